// lbfe_fused_db.cu -- the time step with one cell per thread on 32 x 8
// tiles and the plane copies pipelined two planes deep.
//
// The arithmetic is that of k_fused (lbfe_fused.cu, stages described in
// lbfe_step.cuh); what differs is where the planes wait.  With one staging
// buffer the copy of plane p + 1 can only start once stage M has read plane
// p, and the copy's latency (about 2 us for the 85 KB region of an 8-row
// tile) is then exposed on every plane together with the step's own global
// writes.  Here two staging buffers each take a whole plane (populations,
// the conformation box and, in the reduced forms, the offset densities), so
// the copy of plane p + 2 is in flight while planes p and p + 1 are worked
// on.  To make room (FP32: 2 x 84.5 KB of staging):
//  * the rings hold three planes each: the momentum j of plane p shares the
//    velocity ring (F(q) turns the slot's j(q) into u(q) in place), and the
//    two values that fell out -- the own cell's C and u of plane r - 1 for
//    stage U(r) -- wait in tensor memory (per-thread lanes, like the
//    populations of the collision), written by stages M and F and read back
//    by stage U;
//  * there is no ring of stress scalars: stage F evaluates the prefactor
//    a f and a of Pi = a (f C) - a I at the six face neighbours from the
//    density and conformation rings (the same expression stage M of k_fused
//    stores).
// Shared memory for FP32: rings 57.0 KB + 2 x 82.5 KB = 226 KB.
#include "lbfe_step.cuh"

namespace lbfe {

namespace {

constexpr int DTY = 8;   // tile height of this kernel

// Rings (offsets in floats): rho float2 [3][R2N]; C [3] x float2 [3][R2N]
// ((xx, xy), (yy, yz), (xz, zz)); uj [3] x (float2 [R2N], float [R2N])
// holding j of the newest plane, u of the two before it.
template <int TY>
struct RingDB {
    static constexpr int R2N = Geom<TY>::R2N;
    static_assert(R2N % 4 == 0, "ring alignment");
    static constexpr int RHO = 0, C = 6 * R2N, UJ = C + 18 * R2N;
    static constexpr int FLOATS = UJ + 9 * R2N;
    __device__ static float2 *rho(int s) { return reinterpret_cast<float2 *>(smem() + RHO) + s * R2N; }
    __device__ static float2 *c(int s, int k) { return reinterpret_cast<float2 *>(smem() + C + (s * 3 + k) * 2 * R2N); }
    __device__ static float2 *uxy(int s) { return reinterpret_cast<float2 *>(smem() + UJ + s * 3 * R2N); }
    __device__ static float *uz(int s) { return smem() + UJ + s * 3 * R2N + 2 * R2N; }
};

// Staging: NB buffers, each a whole plane: the populations (box
// BW x (TY+4) x 38 from XPAD cells left of the tile), the conformation (box
// 40 x (TY+4) x 6 from 4 cells left) and, in the reduced forms, the offset
// densities (36 x (TY+4) float2 from 2 cells left); one barrier each.
template <typename T, int TY>
struct StageDB {
    static constexpr int NB = 2;
    static constexpr int XPAD = 16 / (int)sizeof(T);
    static constexpr int BW = 32 + 2 * XPAD, BH = TY + 4;
    static constexpr int POP_PLANE = BW * BH;
    static constexpr u32 POP_BYTES = (u32)(POP_PLANE * 2 * Q * sizeof(T));
    static constexpr int C_PLANE = 40 * BH;
    static constexpr u32 C_OFF = (POP_BYTES + 127u) & ~127u;
    static constexpr u32 C_BYTES = (u32)(C_PLANE * 6 * sizeof(float));
    static constexpr bool DENS = sizeof(T) == 2;
    static constexpr u32 D_OFF = (C_OFF + C_BYTES + 127u) & ~127u;
    static constexpr u32 D_BYTES = DENS ? (u32)(36 * BH * sizeof(float2)) : 0u;
    static constexpr u32 PBUF = (D_OFF + D_BYTES + 127u) & ~127u;
};

template <typename T>
constexpr size_t db_smem_bytes() {
    return sizeof(float) * RingDB<DTY>::FLOATS + 128 + StageDB<T, DTY>::NB * StageDB<T, DTY>::PBUF;
}
static_assert(db_smem_bytes<float>() <= 227 * 1024 - 512, "FP32 staging does not fit");
static_assert(db_smem_bytes<__half>() <= 227 * 1024 - 512, "FP16 staging does not fit");

// TMEM per warp: 256 columns from (warp / 4) * 256 in lane quarter warp % 4:
// [0, 38) and [64, 102) populations of planes of even / odd index; from 128
// four 8-column slots of the own cell's C (plane & 3); from 160 four
// 4-column slots of its u (plane & 3).
constexpr u32 kDbTmemCols = 512;
constexpr u32 kTmC = 128, kTmU = 160;

__device__ __forceinline__ void tm_st1(u32 taddr, float v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(taddr), "r"(__float_as_uint(v)));
}
__device__ __forceinline__ void tm_ld1(u32 taddr, u32 *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r[0]) : "r"(taddr));
}
// Completes pending TMEM loads; the 9 registers pass through the statement.
__device__ __forceinline__ void tm_wait_ld9(u32 *r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]));
}

template <typename T>
__device__ __forceinline__ void m_load_region_db(const StepInst &I, const T *sp, int gx, int gy, u32 n, MCell &m) {
    const float *sc = reinterpret_cast<const float *>(reinterpret_cast<const char *>(sp) + StageDB<T, DTY>::C_OFF);
    using St = StageDB<T, DTY>;
    float2 o = make_float2(0.f, 0.f);
    if (Store<T>::offset) {
        if (St::DENS && I.dens_in)
            o = reinterpret_cast<const float2 *>(reinterpret_cast<const char *>(sp) + St::D_OFF)[gy * 36 + gx];
        else
            o = cell_offsets<T>(I, n);
    }
    const int e = gy * St::BW + gx - 2 + St::XPAD;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        m.ab[i].x = Store<T>::ld_plain(sp + i * St::POP_PLANE + e);
        m.ab[i].y = Store<T>::ld_plain(sp + (Q + i) * St::POP_PLANE + e);
        if (Store<T>::offset) m.ab[i] = fma2(bc(wq(i)), o, m.ab[i]);
    }
    const int ec = gy * 40 + gx + 2;
#pragma unroll
    for (int k = 0; k < 6; ++k) m.c[k] = sc[k * St::C_PLANE + ec];
}

// Stage M for one cell into the ring slot s of its plane: densities, j (in
// the velocity ring), C and the stress scalars.
__device__ __forceinline__ void m_store_db(const StepInst &I, const MCell &m, int idx, int s) {
    using Rg = RingDB<DTY>;
    float2 r = m.ab[0];
#pragma unroll
    for (int i = 1; i < Q; ++i) r = add2(r, m.ab[i]);
    float2 jx = bc(0.f), jy = jx, jz = jx;
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const float2 d = sub2(m.ab[i], m.ab[i + 1]);
        if (cx(i)) jx = cx(i) > 0 ? add2(jx, d) : sub2(jx, d);
        if (cy(i)) jy = cy(i) > 0 ? add2(jy, d) : sub2(jy, d);
        if (cz(i)) jz = cz(i) > 0 ? add2(jz, d) : sub2(jz, d);
    }
    Rg::rho(s)[idx] = r;
    Rg::uxy(s)[idx] = make_float2(jx.x + jx.y, jy.x + jy.y);
    Rg::uz(s)[idx] = jz.x + jz.y;
    Rg::c(s, 0)[idx] = make_float2(m.c[0], m.c[3]);
    Rg::c(s, 1)[idx] = make_float2(m.c[1], m.c[5]);
    Rg::c(s, 2)[idx] = make_float2(m.c[4], m.c[2]);
}

// Stress scalars (a f, a) of Pi = a (f C) - a I at a cell with densities
// rho2 and conformation diagonal (cxx, cyy, czz): a = (eta_P/tau_P) chi,
// chi = rho_visc / rho, f the Peterlin factor of Eq. 2.
__device__ __forceinline__ float2 stress_scalars(const StepInst &I, float2 rho2, float cxx, float cyy, float czz) {
    const float a = I.pi_coef * (I.visc_comp == 0 ? rho2.x : rho2.y) / (rho2.x + rho2.y);
    const float fp = peterlin(I.L2, cxx, cyy, czz);
    return make_float2(a * fp, a);
}

// Stage F for one cell of plane q (ring slots s3 of planes q-1, q, q+1):
// Shan-Chen and polymer forces, and u = (j + F/2)/rho written over j(q).
__device__ __forceinline__ void stage_f_cell_db(const StepInst &I, int idx, const int s3[3], float FA[3],
                                                float FB[3], float u[3], float &rA, float &rB) {
    constexpr int RX = Geom<DTY>::RX;
    using Rg = RingDB<DTY>;
    const float2 *rm = Rg::rho(s3[0]), *rc = Rg::rho(s3[1]), *rp = Rg::rho(s3[2]);
    const float2 r0 = rc[idx];
    rA = r0.x;
    rB = r0.y;
    float sA[3] = {0.f, 0.f, 0.f}, sB[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const int o = cx(i) + cy(i) * RX;
        const float2 a = (cz(i) > 0 ? rp : (cz(i) < 0 ? rm : rc))[idx + o];
        const float2 b = (cz(i) > 0 ? rm : (cz(i) < 0 ? rp : rc))[idx - o];
        const float dA = a.x - b.x, dB = a.y - b.y, w = wq(i);
        if (cx(i)) { sA[0] += cx(i) * w * dB; sB[0] += cx(i) * w * dA; }
        if (cy(i)) { sA[1] += cy(i) * w * dB; sB[1] += cy(i) * w * dA; }
        if (cz(i)) { sA[2] += cz(i) * w * dB; sB[2] += cz(i) * w * dA; }
    }
    float FP[3] = {0.f, 0.f, 0.f};
    if (I.visc_comp >= 0) {
        const float2 *c0 = Rg::c(s3[1], 0), *c1 = Rg::c(s3[1], 1), *c2 = Rg::c(s3[1], 2);
        // the face neighbours' conformation: pairs (xx, xy), (yy, yz), (xz, zz)
        const float2 xp0 = c0[idx + 1], xm0 = c0[idx - 1], xp1 = c1[idx + 1], xm1 = c1[idx - 1];
        const float2 xp2v = c2[idx + 1], xm2v = c2[idx - 1];
        const float2 yp0v = c0[idx + RX], ym0v = c0[idx - RX], yp2v = c2[idx + RX], ym2v = c2[idx - RX];
        const float2 yp1 = c1[idx + RX], ym1 = c1[idx - RX];
        const float2 zp0v = Rg::c(s3[2], 0)[idx], zm0v = Rg::c(s3[0], 0)[idx];
        const float2 zp1v = Rg::c(s3[2], 1)[idx], zm1v = Rg::c(s3[0], 1)[idx];
        const float2 zp2 = Rg::c(s3[2], 2)[idx], zm2 = Rg::c(s3[0], 2)[idx];
        const float2 Ax = stress_scalars(I, rc[idx + 1], xp0.x, xp1.x, xp2v.y);
        const float2 Bx = stress_scalars(I, rc[idx - 1], xm0.x, xm1.x, xm2v.y);
        const float2 Ay = stress_scalars(I, rc[idx + RX], yp0v.x, yp1.x, yp2v.y);
        const float2 By = stress_scalars(I, rc[idx - RX], ym0v.x, ym1.x, ym2v.y);
        const float2 Az = stress_scalars(I, rp[idx], zp0v.x, zp1v.x, zp2.y);
        const float2 Bz = stress_scalars(I, rm[idx], zm0v.x, zm1v.x, zm2.y);
        const float xp2 = xp2v.x, xm2 = xm2v.x;
        const float yp0 = yp0v.y, ym0 = ym0v.y;
        const float zp1 = zp1v.y, zm1 = zm1v.y;
        float gxd = Ax.x * xp0.x - Bx.x * xm0.x;
        float gyd = Ay.x * yp0 - By.x * ym0;
        float gzd = Az.x * zp2.x - Bz.x * zm2.x;
        gxd -= Ax.y - Bx.y;
        FP[0] = 0.5f * (gxd + gyd + gzd);
        gxd = Ax.x * xp0.y - Bx.x * xm0.y;
        gyd = Ay.x * yp1.x - By.x * ym1.x;
        gzd = Az.x * zp1 - Bz.x * zm1;
        gyd -= Ay.y - By.y;
        FP[1] = 0.5f * (gxd + gyd + gzd);
        gxd = Ax.x * xp2 - Bx.x * xm2;
        gyd = Ay.x * yp1.y - By.x * ym1.y;
        gzd = Az.x * zp2.y - Bz.x * zm2.y;
        gzd -= Az.y - Bz.y;
        FP[2] = 0.5f * (gxd + gyd + gzd);
    }
    const float g[3] = {I.gx, I.gy, I.gz};
    const float inv = 1.0f / (rA + rB);
    float2 *uxy = Rg::uxy(s3[1]);
    float *uzp = Rg::uz(s3[1]);
    const float2 jxy = uxy[idx];
    const float j[3] = {jxy.x, jxy.y, uzp[idx]};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        FA[a] = -I.G * rA * sA[a] + (rA * inv) * FP[a] + rA * g[a];
        FB[a] = -I.G * rB * sB[a] + (rB * inv) * FP[a] + rB * g[a];
        u[a] = (j[a] + 0.5f * (FA[a] + FB[a])) * inv;
    }
    uxy[idx] = make_float2(u[0], u[1]);
    uzp[idx] = u[2];
}

// Stage U for the own cell of plane r: ring slots sr (plane r) and sq
// (plane r + 1); the own cell's u and C of plane r - 1 come from tensor
// memory (um, cm).  Same arithmetic as stage_u_cell (first-order upwind).
__device__ __forceinline__ bool stage_u_cell_db(const StepInst &I, int idx, int sr, int sq, int r, const float um[3],
                                                const float cm[6], float cn[6]) {
    constexpr int RX = Geom<DTY>::RX;
    using Rg = RingDB<DTY>;
    const float Uw = I.Uw;
    const int Lz = I.Lz;
    const float2 *uxc = Rg::uxy(sr);
    const float *uzc = Rg::uz(sr);
    const float2 u01 = uxc[idx];
    const float u0[3] = {u01.x, u01.y, uzc[idx]};
    const float2 axp = uxc[idx + 1], axm = uxc[idx - 1], ayp = uxc[idx + RX], aym = uxc[idx - RX];
    const float zxp = uzc[idx + 1], zxm = uzc[idx - 1], zyp = uzc[idx + RX], zym = uzc[idx - RX];
    const float2 up01 = Rg::uxy(sq)[idx];
    const float upn[3] = {up01.x, up01.y, Rg::uz(sq)[idx]};
    const float uxp[3] = {axp.x, axp.y, zxp}, uxm[3] = {axm.x, axm.y, zxm};
    const float uyp[3] = {ayp.x, ayp.y, zyp}, uym[3] = {aym.x, aym.y, zym};
    float Gr[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float uwb = j == 0 ? -Uw : 0.f, uwt = j == 0 ? Uw : 0.f;
        const float uzp = (r == Lz - 1) ? 2.f * uwt - u0[j] : upn[j];
        const float uzm = (r == 0) ? 2.f * uwb - u0[j] : um[j];
        Gr[0][j] = 0.5f * (uxp[j] - uxm[j]);
        Gr[1][j] = 0.5f * (uyp[j] - uym[j]);
        Gr[2][j] = 0.5f * (uzp - uzm);
    }
    auto c_at = [&](int s, int n, float out[6]) {
        const float2 p0 = Rg::c(s, 0)[n], p1 = Rg::c(s, 1)[n], p2 = Rg::c(s, 2)[n];
        out[0] = p0.x; out[1] = p1.x; out[2] = p2.y; out[3] = p0.y; out[4] = p2.x; out[5] = p1.y;
    };
    float c[6];
    c_at(sr, idx, c);
    const int ox = u0[0] > 0.f ? -1 : 1, oy = u0[1] > 0.f ? -RX : RX;
    const float sx = u0[0] > 0.f ? u0[0] : -u0[0], sy = u0[1] > 0.f ? u0[1] : -u0[1];
    const float sz = u0[2] > 0.f ? u0[2] : -u0[2];
    float cx_[6], cy_[6], cz6[6];
    c_at(sr, idx + ox, cx_);
    c_at(sr, idx + oy, cy_);
    if (u0[2] > 0.f) {
#pragma unroll
        for (int q6 = 0; q6 < 6; ++q6) cz6[q6] = cm[q6];
    } else {
        c_at(sq, idx, cz6);
    }
    float adv[6];
#pragma unroll
    for (int q6 = 0; q6 < 6; ++q6) adv[q6] = sx * (c[q6] - cx_[q6]) + sy * (c[q6] - cy_[q6]) + sz * (c[q6] - cz6[q6]);
    const float Cm[3][3] = {{c[0], c[3], c[4]}, {c[3], c[1], c[5]}, {c[4], c[5], c[2]}};
    const float fp = peterlin(I.L2, c[0], c[1], c[2]);
#pragma unroll
    for (int q6 = 0; q6 < 6; ++q6) {
        const int a = q6 < 3 ? q6 : (q6 == 5 ? 1 : 0);
        const int b = q6 < 3 ? q6 : (q6 == 3 ? 1 : 2);
        float st = 0.f;
#pragma unroll
        for (int m = 0; m < 3; ++m) st += Cm[a][m] * Gr[m][b] + Gr[m][a] * Cm[m][b];
        const float relax = (fp * c[q6] - (q6 < 3 ? 1.f : 0.f)) * I.inv_tauP;
        cn[q6] = c[q6] + (-adv[q6] + st - relax);
    }
    return c[0] + c[1] + c[2] < I.L2;
}

// One thread: copy plane `plane` (clamped to the lattice) of item P into the
// staging buffer at dst, completing on bar.
template <typename T>
__device__ __forceinline__ void issue_stage_db(const StepArgs &A, const ItemPos &P, int plane, u32 dst, u32 bar,
                                               u32 go) {
    using St = StageDB<T, DTY>;
    const StepInst &I = A.inst[P.k];
    const int z = min(max(plane, 0), I.Lz - 1);
    const bool dcopy = St::DENS && I.dens_in != nullptr;
    mbar_expect_p(bar, St::POP_BYTES + St::C_BYTES + (dcopy ? St::D_BYTES : 0u), go);
    tma_box4_p(&I.maps->pop, dst, bar, P.bx * 32 - St::XPAD, P.by * DTY - 2, z, go);
    tma_box4_p(&I.maps->c, dst + St::C_OFF, bar, P.bx * 32 - 4, P.by * DTY - 2, z, go);
    if (dcopy) tma_box3_p(&I.maps->dens, dst + St::D_OFF, bar, P.bx * 32 - 2, P.by * DTY - 2, z, go);
}

template <typename T>
__global__ void __launch_bounds__(32 * DTY, 1)
k_fused_db(const __grid_constant__ StepArgs A) {
    constexpr int TY = DTY;
    using Gm = Geom<TY>;
    constexpr int TX = Gm::TX, NT = Gm::NT, RX = Gm::RX, RY = Gm::RY, MH = Gm::MH;
    using St = StageDB<T, TY>;
    using Rg = RingDB<TY>;
    constexpr int NB = St::NB;
    static_assert(MH == 1, "one stage-M halo cell per thread");
    __shared__ u32 s_rows[RY];
    __shared__ u32 s_cols[RX];
    __shared__ u32 s_tmem;
    __shared__ __align__(8) unsigned long long s_bar[NB];   // staging buffer b filled
    __shared__ int s_item[2];

    const int t = threadIdx.x, tx = t & 31, ty = t >> 5;
    const int idx_in = (ty + 2) * RX + (tx + 2);
    const u32 smem_base = smem_addr(lbfe_smem4);
    const u32 buf0 = (smem_base + (u32)(sizeof(float) * Rg::FLOATS) + 127u) & ~127u;
    const char *gen0 = reinterpret_cast<const char *>(lbfe_smem4) - smem_base;   // generic = gen0 + shared address
    u32 par = 0;         // bit b: phase parity of the next completion of buffer b
    // issuing thread (thread 0): bit b of bany = a copy went out on buffer b,
    // of bcnt = the parity of their count (the last one's phase parity is
    // its complement)
    u32 bany = 0, bcnt = 0;
    bool expired = false;

    if (ty == 0) tm_alloc(&s_tmem, kDbTmemCols);
    if (t == 0) {
#pragma unroll
        for (int b = 0; b < NB; ++b) mbar_init(smem_addr(&s_bar[b]));
    }
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const u32 tm_warp = s_tmem + ((u32)(32 * (ty & 3)) << 16) + (u32)((ty >> 2) * 256);

    // Block b starts with item b; further items come from the launch's
    // counter, one ahead.  Plane loads are numbered per block across its
    // items; load k goes to buffer k % NB.
    if (t == 0) {
        s_item[0] = blockIdx.x;
        if ((int)blockIdx.x < A.total_items) {
            const ItemPos P0 = item_pos<TY>(A, blockIdx.x);
            if (A.inst[P0.k].tma) {
#pragma unroll
                for (int b = 0; b < NB; ++b)
                    issue_stage_db<T>(A, P0, P0.z0 - 2 + b, buf0 + (u32)b * St::PBUF, smem_addr(&s_bar[b]), 1u);
                bany = bcnt = (1u << NB) - 1u;
            }
        }
    }
    __syncthreads();
    int slot = 0;
    u32 kload = 0;   // plane loads consumed by this block
    for (int item = s_item[0]; item < A.total_items;) {
        int next_t0 = A.total_items;
        if (t == 0 && A.total_items > (int)gridDim.x) next_t0 = (int)(gridDim.x + atomicAdd(A.work, 1u));
        const ItemPos P = item_pos<TY>(A, item);
        const StepInst &I = A.inst[P.k];
        const int Lx = I.Lx, Ly = I.Ly, Lz = I.Lz;
        const int LxLy = I.LxLy;
        const u32 S = I.S;
        const int bx = P.bx, by = P.by, z0 = P.z0, z1 = P.z1;
        const int x0 = bx * TX - 2, y0 = by * TY - 2;
        const bool tma = I.tma != 0;
        const T *__restrict__ fin = (const T *)I.fin;
        T *__restrict__ fout = (T *)I.fout;
        const float *__restrict__ Cin = I.Cin;
        float *__restrict__ Cout = I.Cout;
        const float Uw = I.Uw;

        __syncthreads();
        if (t < RY) s_rows[t] = (u32)(wrapg(y0 + t, Ly) * Lx);
        if (t < RX) s_cols[t] = (u32)wrapg(x0 + t, Lx);
        __syncthreads();

        const int x = bx * TX + tx, y = by * TY + ty;
        const bool valid = x < Lx && y < Ly;
        const u32 ofs_in = s_rows[ty + 2] + s_cols[tx + 2];
        int dxy[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) dxy[a][b] = (int)(s_rows[ty + 1 + b] + s_cols[tx + 1 + a]) - (int)ofs_in;
        // this thread's stage-M halo cell (threads t < NRING2)
        int h_gx, h_gy;
        ring2_coord<TY>(min(t, Gm::NRING2 - 1), h_gx, h_gy);
        const bool h_on = t < Gm::NRING2;
        const u32 h_ofs = s_rows[h_gy] + s_cols[h_gx];
        const int h_idx = h_gy * RX + h_gx;
        const bool h_dom = (x0 + h_gx) >= 0 && (x0 + h_gx) < Lx && (y0 + h_gy) >= 0 && (y0 + h_gy) < Ly;

        float FA[3], FB[3], uo[3], rAo = 1.f, rBo = 0.f;

        for (int p = z0 - 2; p <= z1 + 1; ++p, ++kload) {
            const int q = p - 1, r = p - 2;
            const int s3[3] = {ring3(q - 1), ring3(q), ring3(q + 1)};   // planes r, q, p
            const u32 pb = kload % (u32)NB;
            const T *stage = reinterpret_cast<const T *>(gen0 + buf0 + pb * St::PBUF);
            // ---------------- stage M(p)
            {
                const u32 pl = (u32)(min(max(p, 0), Lz - 1) * LxLy);
                MCell mh;
                // halo cells across a periodic seam (outside the copied box)
                if (h_on && !(tma && h_dom)) m_load<T>(I, fin, Cin, S, pl + h_ofs, mh);
                if (tma) {
                    if (!expired && !mbar_wait(smem_addr(&s_bar[pb]), (par >> pb) & 1u)) expired = true;
                    par ^= 1u << pb;
                }
                {
                    MCell m;
                    if (tma && valid)
                        m_load_region_db<T>(I, stage, tx + 2, ty + 2, pl + ofs_in, m);
                    else
                        m_load<T>(I, fin, Cin, S, pl + ofs_in, m);
                    m_store_db(I, m, idx_in, s3[2]);
                    tm_store38(tm_warp + (u32)((p & 1) * 64), reinterpret_cast<const float *>(m.ab));
                    // own C of plane p, for stage U(p + 1)
                    const u32 tc = tm_warp + kTmC + (u32)((p & 3) * 8);
                    tm_st4(tc, m.c);
                    tm_st2(tc + 4, m.c + 4);
                }
                if (h_on) {
                    if (tma && h_dom) m_load_region_db<T>(I, stage, h_gx, h_gy, pl + h_ofs, mh);
                    m_store_db(I, mh, h_idx, s3[2]);
                }
            }
            __syncthreads();
            if (t == 0) {
                if (p == z0 - 2) s_item[slot ^ 1] = next_t0;
                // the buffer just read takes the plane NB loads ahead (of this
                // item, else of the next one, whose id this thread took)
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                const u32 go = expired ? 0u : 1u;
                ItemPos Po = P;
                int plane = p + NB;
                bool have = true;
                if (plane > z1 + 1) {
                    have = next_t0 < A.total_items;
                    if (have) {
                        Po = item_pos<TY>(A, next_t0);
                        plane = Po.z0 - 2 + (p + NB - (z1 + 2));
                    }
                }
                if (have && A.inst[Po.k].tma) {
                    issue_stage_db<T>(A, Po, plane, buf0 + pb * St::PBUF, smem_addr(&s_bar[pb]), go);
                    bany |= go << pb;
                    bcnt ^= go << pb;
                }
            }
            // the collision's populations and stage U's own-cell values of
            // plane r - 1 start to come back from TMEM here, ahead of stage F
            const bool doX = q >= z0 && q < z1, doU = r >= z0 && r < z1;
            u32 tr[38], hv[9];
            if (doX || doU) tm_wait_st();
            if (doX) {
                const u32 ta = tm_warp + (u32)((q & 1) * 64);
                tm_ld32(ta, tr);
                tm_ld4(ta + 32, tr + 32);
                tm_ld2(ta + 36, tr + 36);
            }
            if (doU) {
                const u32 tc = tm_warp + kTmC + (u32)(((r - 1) & 3) * 8);
                const u32 tu = tm_warp + kTmU + (u32)(((r - 1) & 3) * 4);
                tm_ld4(tc, hv);
                tm_ld2(tc + 4, hv + 4);
                tm_ld2(tu, hv + 6);
                tm_ld1(tu + 2, hv + 8);
            }
            // ---------------- stage F(q): radius-1 region
            if (q >= max(z0 - 1, 0) && q <= min(z1, Lz - 1)) {
                stage_f_cell_db(I, idx_in, s3, FA, FB, uo, rAo, rBo);
                // own u of plane q, for stage U(q + 1)
                const u32 tu = tm_warp + kTmU + (u32)((q & 3) * 4);
                tm_st2(tu, uo);
                tm_st1(tu + 2, uo[2]);
                for (int h = t; h < Gm::NRING1; h += NT) {
                    int gx, gy;
                    ring1_coord<TY>(h, gx, gy);
                    float a[3], b[3], uu[3], ra, rb;
                    stage_f_cell_db(I, gy * RX + gx, s3, a, b, uu, ra, rb);
                }
            }
            // ---------------- stage X(q): collision + push streaming
            if (doX) {
                tm_wait_ld38(tr);
                float2 fx[Q];
#pragma unroll
                for (int i = 0; i < Q; ++i) fx[i] = make_float2(__uint_as_float(tr[2 * i]), __uint_as_float(tr[2 * i + 1]));
                if (valid) {
                    const u32 nq = (u32)(q * LxLy) + ofs_in;
                    const float rt = rAo + rBo;
                    if (!(rt > 0.f) || uo[0] != uo[0] || uo[1] != uo[1] || uo[2] != uo[2])
                        raise_step_flag(A.status, I, kFlagDiverged);
                    const float om = rt / (3.0f * (rAo * I.nu_A + rBo * I.nu_B) + 0.5f * rt);
                    const bool bottom = q == 0, top = q == Lz - 1;
                    PushOffsets Po;
                    Po.ring[0] = Rg::rho(s3[0]);
                    Po.ring[1] = Rg::rho(s3[1]);
                    Po.ring[2] = Rg::rho(s3[2]);
                    Po.idx = idx_in;
                    Po.own = make_float2(rAo, rBo);
                    Po.track = I.dens_out != nullptr;
                    Po.r0 = make_float2(I.rho0A, I.rho0B);
                    const float2 F2[3] = {make_float2(FA[0], FB[0]), make_float2(FA[1], FB[1]),
                                          make_float2(FA[2], FB[2])};
                    if (bottom || top)
                        collide_push_ab<T, true, RX>(fx, fout, S, Po.own, Po, uo, F2, om, nq, bottom, top, Uw, LxLy,
                                                     dxy);
                    else
                        collide_push_ab<T, false, RX>(fx, fout, S, Po.own, Po, uo, F2, om, nq, false, false, Uw,
                                                      LxLy, dxy);
                    if (Store<T>::offset && Po.track) I.dens_out[nq] = Po.own;
                }
            }
            // ---------------- stage U(r): FENE-P update
            if (doU) {
                tm_wait_ld9(hv);
                if (valid) {
                    const float cm[6] = {__uint_as_float(hv[0]), __uint_as_float(hv[1]), __uint_as_float(hv[2]),
                                         __uint_as_float(hv[3]), __uint_as_float(hv[4]), __uint_as_float(hv[5])};
                    const float um[3] = {__uint_as_float(hv[6]), __uint_as_float(hv[7]), __uint_as_float(hv[8])};
                    float cn[6];
                    if (!stage_u_cell_db(I, idx_in, s3[0], s3[1], r, um, cm, cn))
                        raise_step_flag(A.status, I, kFlagDiverged);
                    const u32 n = (u32)(r * LxLy) + ofs_in;
#pragma unroll
                    for (int q6 = 0; q6 < 6; ++q6) Cout[(u32)(q6 * S + n)] = cn[q6];
                }
            }
            __syncthreads();
        }
        item = s_item[slot ^ 1];
        slot ^= 1;
    }

    if (t == 0 && A.total_items > (int)gridDim.x) release_work_counters(A.work);
    if (expired && t == 0) {
        // copies issued but not waited for may still be in flight: wait,
        // bounded, for the last phase of each barrier before the block's
        // shared memory is released
#pragma unroll
        for (int b = 0; b < NB; ++b)
            if ((bany >> b) & 1u) mbar_wait(smem_addr(&s_bar[b]), ((bcnt >> b) & 1u) ^ 1u);
    }
    if (expired) atomicOr(A.status, kFlagTimeout);
    tm_wait_st();
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    if (ty == 0) tm_dealloc(s_tmem, kDbTmemCols);
}

template <typename T>
cudaError_t db_launch_t(const StepArgs &a, int grid, cudaStream_t st) {
    k_fused_db<T><<<grid, Geom<DTY>::NT, db_smem_bytes<T>(), st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t db_prep_t(int *bps) {
    const size_t smem = db_smem_bytes<T>();
    cudaError_t e = cudaFuncSetAttribute(k_fused_db<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int b = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_fused_db<T>, Geom<DTY>::NT, smem);
    if (e != cudaSuccess) return e;
    // every block allocates all 512 TMEM columns of its SM
    *bps = b < 1 ? b : 1;
    return cudaSuccess;
}

}  // namespace

cudaError_t step_db_launch(const StepArgs &a, int grid, int precision, cudaStream_t st) {
    switch (precision) {
        case LBFE_FP16_OFFSET: return db_launch_t<__half>(a, grid, st);
        case LBFE_BF16_OFFSET: return db_launch_t<__nv_bfloat16>(a, grid, st);
        default: return db_launch_t<float>(a, grid, st);
    }
}

cudaError_t step_db_prepare(int precision, int *blocks_per_sm) {
    switch (precision) {
        case LBFE_FP16_OFFSET: return db_prep_t<__half>(blocks_per_sm);
        case LBFE_BF16_OFFSET: return db_prep_t<__nv_bfloat16>(blocks_per_sm);
        default: return db_prep_t<float>(blocks_per_sm);
    }
}

}  // namespace lbfe
