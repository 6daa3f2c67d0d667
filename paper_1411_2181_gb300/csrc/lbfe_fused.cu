// lbfe_fused.cu -- one time step of the hybrid LBM / FENE-P method (Sec. 2)
// in a single persistent kernel that reads every population and conformation
// component once and writes it once.
//
// Work decomposition.  A work item is a column tile of 32 x TY cells in the
// x-y plane over a chunk [z0, z1) of planes of one instance; blocks stride
// over the work items of all instances of a batch.  Inside an item the block
// marches along z with shared-memory rings holding, per plane, the fields the
// stencils need:
//   stage M(p)    moments rho_A, rho_B, j and the polymer stress
//                 Pi = (eta_P/tau_P) chi (f C - I) of plane p on the
//                 radius-2 region (36 x (TY+4) cells; the halo is recomputed
//                 from the populations of the neighbouring columns);
//   stage F(p-1)  Shan-Chen force (radius-1 densities), polymer force
//                 div Pi, the Guo velocity u = (j + F/2)/rho on the radius-1
//                 region (34 x (TY+2));
//   stage X(p-1)  BGK + Guo collision of the tile's own cells and push
//                 streaming with halfway bounce-back on the moving walls;
//   stage U(p-2)  FENE-P update of C (Eq. 2/4): central grad u from the
//                 velocity ring, first-order upwind u.grad C from the
//                 conformation ring.
// The collision of plane p-1 needs the densities of plane p (Shan-Chen); the
// C update of plane p-2 needs the velocity of plane p-1, hence the lags.
// Three block barriers per plane: after stage M, after stage X (stage X
// needs only its own cell's forces, so it runs before the barrier that
// stage U needs) and after stage U.
// Planes beyond a wall are loaded as the adjacent plane (mirror ghosts of
// rho, C and Pi); the velocity ghost 2 U_wall - u is applied in stage U.
#include "lbfe_internal.cuh"

namespace lbfe {

namespace {

template <int TY>
struct Geom {
    static constexpr int TX = 32;
    static constexpr int NT = TX * TY;                 // threads = tile cells
    static constexpr int RX = TX + 4, RY = TY + 4;     // radius-2 region
    static constexpr int R2N = RX * RY;
    static constexpr int NRING1 = 2 * (RX - 2) + 2 * TY;  // radius-1 cells outside the tile
    // rings: rho (float2) x3, stress scalars (a f, a) x3, j 3x2, C 6x4, u 3x3
    static constexpr int FLOATS = (2 * 3 + 2 * 3 + 6 + 24 + 9) * R2N;
};

// Ring slot of plane p (p >= -4) in rings of 2, 3 and 4 planes.
__device__ __forceinline__ int ring2(int p) { return (p + 12) & 1; }
__device__ __forceinline__ int ring3(int p) { return (p + 12) % 3; }
__device__ __forceinline__ int ring4(int p) { return (p + 12) & 3; }
__device__ __forceinline__ int wrapg(int a, int L) { a %= L; return a < 0 ? a + L : a; }

// symmetric-tensor slot of (a, b): xx, yy, zz, xy, xz, yz
__host__ __device__ constexpr int symk(int a, int b) {
    return a == b ? a : ((a + b) == 1 ? 3 : ((a + b) == 2 ? 4 : 5));
}

template <typename T>
__device__ __forceinline__ float ldpop(const T *p, float add) {
    float v = Store<T>::ld(p);
    if (Store<T>::offset) v += add;
    return v;
}

// Ring cell h (0 <= h < NRING1) of the radius-1 region.
template <int TY>
__device__ __forceinline__ void ring1_coord(int h, int &gx, int &gy) {
    using Gm = Geom<TY>;
    if (h < 2 * (Gm::RX - 2)) {
        const int rr = h / (Gm::RX - 2);
        gx = 1 + (h - rr * (Gm::RX - 2));
        gy = rr == 0 ? 1 : Gm::RY - 2;
    } else {
        const int h2 = h - 2 * (Gm::RX - 2);
        const int cc = h2 / TY;
        gy = 2 + (h2 - cc * TY);
        gx = cc == 0 ? 1 : Gm::RX - 2;
    }
}

typedef unsigned int u32;

// Shared-memory rings (offsets in floats from the dynamic shared base):
//   rho  float2 [3][R2N]          densities rho_A, rho_B
//   pi   float  [3][2][R2N]       a f and a of Pi = a (f C) - a I, a = (eta_P/tau_P) chi
//   j    float  [2][3][R2N]       momentum
//   c    float  [4][6][R2N]       conformation
//   u    float  [3][3][R2N]       velocity
template <int TY>
struct Ring {
    static constexpr int R2N = Geom<TY>::R2N;
    static constexpr int RHO = 0, PI = 6 * R2N, J = PI + 6 * R2N, C = J + 6 * R2N, U = C + 24 * R2N;
};

extern __shared__ float4 lbfe_smem4[];
__device__ __forceinline__ float *smem() { return reinterpret_cast<float *>(lbfe_smem4); }

// Stage M inputs of one cell: its 38 populations and 6 conformation components.
struct MCell {
    float f[2 * Q];
    float c[6];
};

// Cell offsets are 32-bit: an instance holds at most 2^26 cells, so every
// field offset (s*19 + i)*S + n stays below 2^32.
template <typename T>
__device__ __forceinline__ void m_load(const InstDev &I, const T *__restrict__ fin, const float *__restrict__ Cin,
                                       u32 S, u32 n, int cur, MCell &m) {
    const float2 od = offset_dens<T>(I, cur, n);
    const float ra0 = od.x, rb0 = od.y;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        m.f[i] = ldpop(fin + (u32)(i * S + n), wq(i) * ra0);
        m.f[Q + i] = ldpop(fin + (u32)((Q + i) * S + n), wq(i) * rb0);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) m.c[k] = __ldg(Cin + (u32)(k * S + n));
}

// Stage M for one cell: moments, stress scalars and conformation into the
// ring slots of its plane.
template <int TY>
__device__ __forceinline__ void m_store(const InstDev &I, const MCell &m, int idx, int s3, int s2, int s4) {
    // s3: rho / stress slot, s2: j slot, s4: C slot of the plane
    constexpr int R2N = Geom<TY>::R2N;
    using Rg = Ring<TY>;
    float2 *rho_s = reinterpret_cast<float2 *>(smem() + Rg::RHO) + s3 * R2N;
    float *pi_s = smem() + Rg::PI + s3 * 2 * R2N;
    float *j_s = smem() + Rg::J + s2 * 3 * R2N;
    float *c_s = smem() + Rg::C + s4 * 6 * R2N;
    float rA = 0.f, rB = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) { rA += m.f[i]; rB += m.f[Q + i]; }
    // momentum from opposite-pair differences (exact in FP32 per pair)
    float jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const float d = (m.f[i] - m.f[i + 1]) + (m.f[Q + i] - m.f[Q + i + 1]);
        if (cx(i)) jx += cx(i) * d;
        if (cy(i)) jy += cy(i) * d;
        if (cz(i)) jz += cz(i) * d;
    }
    rho_s[idx] = make_float2(rA, rB);
    j_s[idx] = jx;
    j_s[R2N + idx] = jy;
    j_s[2 * R2N + idx] = jz;
#pragma unroll
    for (int k = 0; k < 6; ++k) c_s[k * R2N + idx] = m.c[k];
    float a = 0.f, fp = 1.f;
    if (I.visc_comp >= 0) {
        a = I.pi_coef * (I.visc_comp == 0 ? rA : rB) / (rA + rB);
        fp = peterlin(I.L2, m.c[0], m.c[1], m.c[2]);
    }
    pi_s[idx] = a * fp;
    pi_s[R2N + idx] = a;
}

// Ring slots of the planes one iteration touches (q = p - 1, r = p - 2).
struct Slots {
    int r3[3];   // rho / stress / u slots of planes q-1, q, q+1
    int ur[3];   // u slots of planes r-1, r, r+1 (= q-2, q-1, q)
    int cf[3];   // C slots of planes q-1, q, q+1 (stage F)
    int cu[3];   // C slots of planes r-1, r, r+1 (stage U)
    int j3;      // j slot of plane q (ring of 2)
};

// Stage F for one cell of plane q: Shan-Chen and polymer forces and the
// velocity.  Writes u to the ring; returns the per-component total forces,
// u and the densities.
template <int TY>
__device__ __forceinline__ void stage_f_cell(const InstDev &I, int idx, const Slots &L, float FA[3], float FB[3],
                                             float u[3], float &rA, float &rB) {
    constexpr int R2N = Geom<TY>::R2N, RX = Geom<TY>::RX;
    using Rg = Ring<TY>;
    const float2 *rho0 = reinterpret_cast<const float2 *>(smem() + Rg::RHO);
    const float2 *rm = rho0 + L.r3[0] * R2N, *rc = rho0 + L.r3[1] * R2N, *rp = rho0 + L.r3[2] * R2N;
    const float2 r0 = rc[idx];
    rA = r0.x;
    rB = r0.y;
    // Shan-Chen with opposite neighbours in pairs: w_i c_i (rho(x + c_i) - rho(x - c_i))
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
    // polymer force F_P,a = sum_b (Pi_ba(x + e_b) - Pi_ba(x - e_b))/2 with
    // Pi_ba = (a f) C_ba - a delta_ba
    float FP[3] = {0.f, 0.f, 0.f};
    if (I.visc_comp >= 0) {
        const float *sm_ = smem() + Rg::PI + L.r3[0] * 2 * R2N;
        const float *sc_ = smem() + Rg::PI + L.r3[1] * 2 * R2N;
        const float *sp_ = smem() + Rg::PI + L.r3[2] * 2 * R2N;
        const float *cm = smem() + Rg::C + L.cf[0] * 6 * R2N;
        const float *cc = smem() + Rg::C + L.cf[1] * 6 * R2N;
        const float *cp = smem() + Rg::C + L.cf[2] * 6 * R2N;
        const float afxp = sc_[idx + 1], afxm = sc_[idx - 1], afyp = sc_[idx + RX], afym = sc_[idx - RX];
        const float afzp = sp_[idx], afzm = sm_[idx];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float gxd = afxp * cc[symk(0, a) * R2N + idx + 1] - afxm * cc[symk(0, a) * R2N + idx - 1];
            float gyd = afyp * cc[symk(1, a) * R2N + idx + RX] - afym * cc[symk(1, a) * R2N + idx - RX];
            float gzd = afzp * cp[symk(2, a) * R2N + idx] - afzm * cm[symk(2, a) * R2N + idx];
            if (a == 0) gxd -= sc_[R2N + idx + 1] - sc_[R2N + idx - 1];
            if (a == 1) gyd -= sc_[R2N + idx + RX] - sc_[R2N + idx - RX];
            if (a == 2) gzd -= sp_[R2N + idx] - sm_[R2N + idx];
            FP[a] = 0.5f * (gxd + gyd + gzd);
        }
    }
    const float g[3] = {I.gx, I.gy, I.gz};
    const float inv = 1.0f / (rA + rB);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        FA[a] = -I.G * rA * sA[a] + (rA * inv) * FP[a] + rA * g[a];
        FB[a] = -I.G * rB * sB[a] + (rB * inv) * FP[a] + rB * g[a];
        u[a] = (smem()[Rg::J + L.j3 * 3 * R2N + a * R2N + idx] + 0.5f * (FA[a] + FB[a])) * inv;
        smem()[Rg::U + L.r3[1] * 3 * R2N + a * R2N + idx] = u[a];
    }
}

// Offsets of the reduced storage forms at the destination of a push:
// the destination cell's densities of this step (from the density ring of
// planes q-1, q, q+1), or the constant offsets when densities are not
// tracked.
struct PushOffsets {
    const float2 *ring[3];   // density ring slots of planes q-1, q, q+1
    int idx;                 // ring index of the pushing cell
    float own[2];            // the pushing cell's densities
    bool track;
    float r0[2];             // constant offsets
};

template <int RX>
__device__ __forceinline__ float push_offset(const PushOffsets &P, int s, int d, bool wall) {
    if (!P.track) return P.r0[s];
    if (wall) return P.own[s];
    const float2 v = P.ring[cz(d) + 1][P.idx + cx(d) + cy(d) * RX];
    return s == 0 ? v.x : v.y;
}

// Store post-collision population d of the cell at offset n into its
// streamed position x + c_d.  With WALLS, a population whose target lies
// beyond a wall returns into the cell as the opposite direction (halfway
// bounce-back) with the moving-wall term -6 w_d rho_s (c_d . U_wall).
template <typename T, bool WALLS, int RX>
__device__ __forceinline__ void push_one(T *__restrict__ fdst, u32 S, int s, int d, float v, float rs,
                                         const PushOffsets &P, u32 n, bool bottom, bool top, float Uw, int LxLy,
                                         const int dxy[3][3]) {
    int dir = d;
    u32 dst = n + (u32)(cz(d) * LxLy + dxy[cx(d) + 1][cy(d) + 1]);
    bool wall = false;
    if (WALLS && ((cz(d) < 0 && bottom) || (cz(d) > 0 && top))) {
        v -= 6.f * wq(d) * rs * (float)cx(d) * (cz(d) < 0 ? -Uw : Uw);
        dir = opp(d);
        dst = n;
        wall = true;
    }
    if (Store<T>::offset) v -= wq(d) * push_offset<RX>(P, s, d, wall);
    Store<T>::st(fdst + (u32)((s * Q + dir) * S + dst), v);
}

// BGK + Guo collision of one component at one cell and push streaming of
// its 19 populations.  Opposite directions share the symmetric parts:
//   f^eq_{i,-i} = w rho (1 + 9/2 (c.u)^2 - 3/2 u.u) +- 3 w rho (c.u)
//   S_{i,-i}    = (1 - 1/2tau) w (9 (c.u)(c.F) - 3 u.F) +- 3 (1 - 1/2tau) w (c.F)
template <typename T, bool WALLS, int RX>
__device__ __forceinline__ void collide_push(const float *fv, T *__restrict__ fdst, u32 S, int s, float rs,
                                             const PushOffsets &P, const float u[3], const float F[3], float om, u32 n,
                                             bool bottom, bool top, float Uw, int LxLy, const int dxy[3][3]) {
    const float omc = 1.0f - om, pref = 1.0f - 0.5f * om;
    const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const float uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
    const float base0 = rs * (1.f - 1.5f * uu);   // rho (1 - 3/2 u.u)
    const float srcb = -3.f * uF * pref;           // (1 - 1/2tau)(-3 u.F)
    {
        float v = omc * fv[0] + wq(0) * (om * base0 + srcb);
        if (Store<T>::offset) v -= wq(0) * (P.track ? P.own[s] : P.r0[s]);
        Store<T>::st(fdst + (u32)(s * Q * S + n), v);
    }
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const float w = wq(i);
        const float cu = cx(i) * u[0] + cy(i) * u[1] + cz(i) * u[2];
        const float cF = cx(i) * F[0] + cy(i) * F[1] + cz(i) * F[2];
        const float sym = w * (om * (base0 + 4.5f * rs * cu * cu) + srcb + 9.f * pref * cu * cF);
        const float anti = w * (om * 3.f * rs * cu + 3.f * pref * cF);
        push_one<T, WALLS, RX>(fdst, S, s, i, omc * fv[i] + (sym + anti), rs, P, n, bottom, top, Uw, LxLy, dxy);
        push_one<T, WALLS, RX>(fdst, S, s, i + 1, omc * fv[i + 1] + (sym - anti), rs, P, n, bottom, top, Uw, LxLy,
                               dxy);
    }
}

}  // namespace

template <typename T, int TY>
__global__ void __launch_bounds__(32 * TY, TY >= 16 ? 1 : (TY >= 8 ? 2 : 3))
k_fused(const InstDev *__restrict__ insts, const int *__restrict__ item_off, int n_inst, int total_items,
        int cur, unsigned *status) {
    using Gm = Geom<TY>;
    constexpr int TX = Gm::TX, NT = Gm::NT, RX = Gm::RX, RY = Gm::RY, R2N = Gm::R2N;
    constexpr int MR = (R2N + NT - 1) / NT;   // stage-M rounds per thread
    using Rg = Ring<TY>;
    __shared__ u32 s_rows[RY];   // in-plane offsets of the radius-2 rows (wrapped)
    __shared__ u32 s_cols[RX];   // x of the radius-2 columns (wrapped)

    const int t = threadIdx.x, tx = t & 31, ty = t >> 5;
    const int idx_in = (ty + 2) * RX + (tx + 2);

    for (int item = blockIdx.x; item < total_items; item += gridDim.x) {
        const int k = find_inst(item_off, n_inst, item);
        const InstDev &I = insts[k];
        const int Lx = I.Lx, Ly = I.Ly, Lz = I.Lz;
        const int LxLy = Lx * Ly;
        const u32 S = (u32)I.S;
        int local = item - __ldg(item_off + k);
        const int bx = local % I.ntx;
        local /= I.ntx;
        const int by = local % I.nty;
        const int zi = local / I.nty;
        const int z0 = zi * I.zc, z1 = min(Lz, z0 + I.zc);
        const int x0 = bx * TX - 2, y0 = by * TY - 2;
        const T *__restrict__ fin = (const T *)I.f[cur];
        T *__restrict__ fout = (T *)I.f[cur ^ 1];
        const float *__restrict__ Cin = I.C[cur];
        float *__restrict__ Cout = I.C[cur ^ 1];
        const float Uw = I.Uw;

        __syncthreads();  // previous item done with the row/column tables
        if (t < RY) s_rows[t] = (u32)(wrapg(y0 + t, Ly) * Lx);
        if (t < RX) s_cols[t] = (u32)wrapg(x0 + t, Lx);
        __syncthreads();

        // own cell and the offsets of its 3 x 3 in-plane neighbourhood
        const int x = bx * TX + tx, y = by * TY + ty;
        const bool valid = x < Lx && y < Ly;
        const u32 ofs_in = s_rows[ty + 2] + s_cols[tx + 2];
        int dxy[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) dxy[a][b] = (int)(s_rows[ty + 1 + b] + s_cols[tx + 1 + a]) - (int)ofs_in;
        // in-plane offsets of this thread's stage-M cells (i = t + r NT)
        u32 om_ofs[MR];
#pragma unroll
        for (int r = 0; r < MR; ++r) {
            const int i = min(t + r * NT, R2N - 1), gy = i / RX;
            om_ofs[r] = s_rows[gy] + s_cols[i - gy * RX];
        }

        float FA[3], FB[3], uo[3], rAo = 1.f, rBo = 0.f;

        for (int p = z0 - 2; p <= z1 + 1; ++p) {
            const int q = p - 1, r = p - 2;
            Slots L;
            L.r3[0] = ring3(q - 1);
            L.r3[1] = ring3(q);
            L.r3[2] = ring3(q + 1);
            L.ur[0] = ring3(q - 2);
            L.ur[1] = L.r3[0];
            L.ur[2] = L.r3[1];
            L.cf[0] = ring4(q - 1);
            L.cf[1] = ring4(q);
            L.cf[2] = ring4(q + 1);
            L.cu[0] = ring4(q - 2);
            L.cu[1] = L.cf[0];
            L.cu[2] = L.cf[1];
            L.j3 = ring2(q);

            // ---------------- stage M(p): radius-2 region of plane clamp(p)
            {
                const u32 pl = (u32)(min(max(p, 0), Lz - 1) * LxLy);
#pragma unroll
                for (int rr = 0; rr < MR; ++rr) {
                    const int i = t + rr * NT;
                    if (rr * NT + NT <= R2N || i < R2N) {
                        MCell m;
                        m_load<T>(I, fin, Cin, S, pl + om_ofs[rr], cur, m);
                        m_store<TY>(I, m, i, L.r3[2], ring2(p), L.cf[2]);
                    }
                }
            }
            __syncthreads();
            // ---------------- stage F(q): radius-1 region
            if (q >= max(z0 - 1, 0) && q <= min(z1, Lz - 1)) {
                stage_f_cell<TY>(I, idx_in, L, FA, FB, uo, rAo, rBo);
                for (int h = t; h < Gm::NRING1; h += NT) {
                    int gx, gy;
                    ring1_coord<TY>(h, gx, gy);
                    float a[3], b[3], uu[3], ra, rb;
                    stage_f_cell<TY>(I, gy * RX + gx, L, a, b, uu, ra, rb);
                }
            }
            // ---------------- stage X(q): collision + push streaming (own cell only:
            // needs no barrier after stage F)
            if (q >= z0 && q < z1 && valid) {
                const u32 nq = (u32)(q * LxLy) + ofs_in;
                const float2 od = offset_dens<T>(I, cur, nq);
                float fx[2 * Q];
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    fx[i] = ldpop(fin + (long long)i * S + nq, wq(i) * od.x);
                    fx[Q + i] = ldpop(fin + (long long)(Q + i) * S + nq, wq(i) * od.y);
                }
                const float rt = rAo + rBo;
                if (!(rt > 0.f) || uo[0] != uo[0] || uo[1] != uo[1] || uo[2] != uo[2])
                    raise_flag(status, I, kFlagDiverged);
                const float nu = (rAo * I.nu_A + rBo * I.nu_B) / rt;
                const float om = 1.0f / (3.0f * nu + 0.5f);
                const bool bottom = q == 0, top = q == Lz - 1;
                PushOffsets P;
                const float2 *rho_s = reinterpret_cast<const float2 *>(smem() + Rg::RHO);
                P.ring[0] = rho_s + L.r3[0] * R2N;
                P.ring[1] = rho_s + L.r3[1] * R2N;
                P.ring[2] = rho_s + L.r3[2] * R2N;
                P.idx = idx_in;
                P.own[0] = rAo;
                P.own[1] = rBo;
                P.track = I.dens[0] != nullptr;
                P.r0[0] = I.rho0[0];
                P.r0[1] = I.rho0[1];
                collide_push<T, true, RX>(fx, fout, S, 0, rAo, P, uo, FA, om, nq, bottom, top, Uw, LxLy, dxy);
                collide_push<T, true, RX>(fx + Q, fout, S, 1, rBo, P, uo, FB, om, nq, bottom, top, Uw, LxLy, dxy);
                // this step's densities: the offsets of the state just written
                if (Store<T>::offset && P.track) I.dens[cur][nq] = make_float2(rAo, rBo);
            }
            __syncthreads();  // u of plane q complete on the radius-1 region
            // ---------------- stage U(r): FENE-P update, Eq. 2 (Eq. 4)
            if (r >= z0 && r < z1 && valid) {
                const float *um = smem() + Rg::U + L.ur[0] * 3 * R2N;
                const float *uc = smem() + Rg::U + L.ur[1] * 3 * R2N;
                const float *up = smem() + Rg::U + L.ur[2] * 3 * R2N;
                const float *cm = smem() + Rg::C + L.cu[0] * 6 * R2N;
                const float *cc = smem() + Rg::C + L.cu[1] * 6 * R2N;
                const float *cp = smem() + Rg::C + L.cu[2] * 6 * R2N;
                const int i0 = idx_in;
                float u0[3], Gr[3][3];
#pragma unroll
                for (int j = 0; j < 3; ++j) u0[j] = uc[j * R2N + i0];
                // grad u by central differences, u_ghost = 2 U_wall - u at the walls
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const float uwb = j == 0 ? -Uw : 0.f, uwt = j == 0 ? Uw : 0.f;
                    const float uzp = (r == Lz - 1) ? 2.f * uwt - u0[j] : up[j * R2N + i0];
                    const float uzm = (r == 0) ? 2.f * uwb - u0[j] : um[j * R2N + i0];
                    Gr[0][j] = 0.5f * (uc[j * R2N + i0 + 1] - uc[j * R2N + i0 - 1]);
                    Gr[1][j] = 0.5f * (uc[j * R2N + i0 + RX] - uc[j * R2N + i0 - RX]);
                    Gr[2][j] = 0.5f * (uzp - uzm);
                }
                float c[6];
#pragma unroll
                for (int q6 = 0; q6 < 6; ++q6) c[q6] = cc[q6 * R2N + i0];
                // first-order upwind u . grad C (C mirrored at the walls)
                const int ox = u0[0] > 0.f ? -1 : 1, oy = u0[1] > 0.f ? -RX : RX;
                const float sx = u0[0] > 0.f ? u0[0] : -u0[0], sy = u0[1] > 0.f ? u0[1] : -u0[1];
                const float sz = u0[2] > 0.f ? u0[2] : -u0[2];
                const float *cz_ = u0[2] > 0.f ? cm : cp;
                float adv[6];
#pragma unroll
                for (int q6 = 0; q6 < 6; ++q6)
                    adv[q6] = sx * (c[q6] - cc[q6 * R2N + i0 + ox]) + sy * (c[q6] - cc[q6 * R2N + i0 + oy]) +
                              sz * (c[q6] - cz_[q6 * R2N + i0]);
                const float Cm[3][3] = {{c[0], c[3], c[4]}, {c[3], c[1], c[5]}, {c[4], c[5], c[2]}};
                const float fp = peterlin(I.L2, c[0], c[1], c[2]);
                const u32 n = (u32)(r * LxLy) + ofs_in;
#pragma unroll
                for (int q6 = 0; q6 < 6; ++q6) {
                    const int a = q6 < 3 ? q6 : (q6 == 5 ? 1 : 0);
                    const int b = q6 < 3 ? q6 : (q6 == 3 ? 1 : 2);
                    float st = 0.f;
#pragma unroll
                    for (int m = 0; m < 3; ++m) st += Cm[a][m] * Gr[m][b] + Gr[m][a] * Cm[m][b];
                    const float relax = (fp * c[q6] - (q6 < 3 ? 1.f : 0.f)) * I.inv_tauP;
                    Cout[(u32)(q6 * S + n)] = c[q6] + (-adv[q6] + st - relax);
                }
                if (!(c[0] + c[1] + c[2] < I.L2)) raise_flag(status, I, kFlagDiverged);
            }
            __syncthreads();  // stage U done with the rings before stage M(p+1)
        }
    }
}

// ---------------------------------------------------------------- host side
template <typename T, int TY>
static cudaError_t fused_t(const LaunchCtx &c, int cur) {
    const size_t smem = sizeof(float) * Geom<TY>::FLOATS;
    k_fused<T, TY><<<c.fused_grid, Geom<TY>::NT, smem, c.stream>>>(c.inst_dev, c.item_off, c.n, c.total_items,
                                                                    cur, c.status);
    return cudaGetLastError();
}

template <int TY>
static cudaError_t fused_ty(const LaunchCtx &c, int cur) {
    switch (c.precision) {
        case LBFE_FP16_OFFSET: return fused_t<__half, TY>(c, cur);
        case LBFE_BF16_OFFSET: return fused_t<__nv_bfloat16, TY>(c, cur);
        default: return fused_t<float, TY>(c, cur);
    }
}

cudaError_t launch_fused(const LaunchCtx &c, int cur) {
    switch (c.tile_y) {
        case 4: return fused_ty<4>(c, cur);
        case 16: return fused_ty<16>(c, cur);
        default: return fused_ty<8>(c, cur);
    }
}

size_t fused_smem_bytes(int tile_y) {
    switch (tile_y) {
        case 4: return sizeof(float) * Geom<4>::FLOATS;
        case 16: return sizeof(float) * Geom<16>::FLOATS;
        default: return sizeof(float) * Geom<8>::FLOATS;
    }
}

template <typename T, int TY>
static cudaError_t prep_t(int *bps) {
    const size_t smem = sizeof(float) * Geom<TY>::FLOATS;
    cudaError_t e = cudaFuncSetAttribute(k_fused<T, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_fused<T, TY>, Geom<TY>::NT, smem);
}

template <int TY>
static cudaError_t prep_ty(int precision, int *bps) {
    switch (precision) {
        case LBFE_FP16_OFFSET: return prep_t<__half, TY>(bps);
        case LBFE_BF16_OFFSET: return prep_t<__nv_bfloat16, TY>(bps);
        default: return prep_t<float, TY>(bps);
    }
}

cudaError_t fused_prepare(int tile_y, int precision, int *blocks_per_sm) {
    switch (tile_y) {
        case 4: return prep_ty<4>(precision, blocks_per_sm);
        case 16: return prep_ty<16>(precision, blocks_per_sm);
        default: return prep_ty<8>(precision, blocks_per_sm);
    }
}

}  // namespace lbfe
