// lbfe_fused.cu -- the time-step kernel with one cell per thread (tiles of
// 32 x TY cells, TY in {8, 12, 16}), and the host side of both step kernels:
// launch descriptors, TMA tensor maps and the grouping of a batch into
// launches.  The stage structure is described in lbfe_step.cuh.
#include <cstring>
#include <mutex>

#include "lbfe_step.cuh"

namespace lbfe {

template <typename T, int TY, bool ADV2 = false>
__global__ void __launch_bounds__(32 * TY, 1)
k_fused(const __grid_constant__ StepArgs A) {
    using Gm = Geom<TY>;
    constexpr int TX = Gm::TX, NT = Gm::NT, RX = Gm::RX, RY = Gm::RY, R2N = Gm::R2N, MH = Gm::MH;
    using St = Stage<T, TY>;
    using Rg = Ring<TY>;
    // interior planes take a push without the bounce-back selection where
    // registers allow the second copy of the collision (not at 16 rows)
    constexpr bool kSplitWalls = TY <= 12;
    // the collision's TMEM loads are issued before stage F where registers
    // allow holding them through it
    constexpr bool kEarlyTmem = TY <= 8;
    __shared__ u32 s_rows[RY];   // in-plane offsets of the radius-2 rows (wrapped)
    __shared__ u32 s_cols[RX];   // x of the radius-2 columns (wrapped)
    __shared__ u32 s_tmem;       // TMEM base address of the block
    __shared__ __align__(8) unsigned long long s_bar;   // TMA completion barrier of the staging buffer
    // every thread has read what it needs from the staging buffer (NT arrivals per plane)
    __shared__ __align__(8) unsigned long long s_empty;

    const int t = threadIdx.x, tx = t & 31, ty = t >> 5;
    const int idx_in = (ty + 2) * RX + (tx + 2);
    // staging buffer for the TMA boxes: after the rings, 128-byte aligned
    const u32 smem_base = smem_addr(lbfe_smem4);
    const u32 stage_addr = (smem_base + (u32)(sizeof(float) * Gm::FLOATS) + 127u) & ~127u;
    const char *stage0 = reinterpret_cast<const char *>(lbfe_smem4) + (stage_addr - smem_base);
    const u32 bar = smem_addr(&s_bar), ebar = smem_addr(&s_empty);
    // Early issue (FP32, 8-row tiles, where the plane copy is the critical
    // path): the next plane's copy starts as soon as every thread has read
    // its cells from the staging buffer, issued by lane 0 of the last warp
    // (which has no halo cells in stage M), instead of by thread 0 after
    // the stage-M barrier.  Measured on 192 x 96 x 80: 158 -> 148 us per
    // step at 32 x 8 (142 us with the staged halo cell read before the own
    // cell); slower for the other shapes (140 -> 160 us at 32 x 12).
    constexpr bool kEarlyIssue = TY == 8 && sizeof(T) == 4;
    constexpr int kIssuer = kEarlyIssue ? NT - 32 : 0;
    static_assert(!St::REGION || MH == 1, "one stage-M halo cell per thread");
    u32 parity = 0;                  // phase parity of the next copy to wait for
    u32 eparity = 0;                 // phase parity of the next 'buffer read' (issuer)
    u32 issued = 0;                  // copies issued (issuer)
    // this thread's wait expired: it waits for no further copy, and the
    // issuer issues none (at most one copy stays outstanding)
    bool expired = false;

    if (ty == 0) tm_alloc(&s_tmem, Gm::TMEM_COLS);
    if (t == 0) {
        mbar_init(bar);
        mbar_init_count(ebar, NT);
    }
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    // this warp's TMEM slot: lane quarter ty % 4, columns (ty / 4) * 128
    const u32 tm_warp = s_tmem + ((u32)(32 * (ty & 3)) << 16) + (u32)((ty >> 2) * 128);

    // Block b starts with item b (neighbouring tiles on neighbouring blocks,
    // which share their halos through L2); further items come from the
    // launch's counter, one ahead: the next item is known while the current
    // one runs, so that its first plane can be copied early, and blocks
    // that finish early take more items.
    __shared__ int s_item[2];
    if (t == 0) s_item[0] = blockIdx.x;
    // the first plane of the block's first item
    if (t == kIssuer && (int)blockIdx.x < A.total_items) {
        const ItemPos P0 = item_pos<TY>(A, blockIdx.x);
        if (A.inst[P0.k].tma) {
            issue_plane<T, TY>(A, P0, P0.z0 - 2, stage_addr, bar);
            ++issued;
        }
    }
    __syncthreads();
    int slot = 0;
    for (int item = s_item[0]; item < A.total_items;) {
        // the next item: taken now, published after the first stage M (the
        // item-start barriers do not wait for the atomic)
        // (a launch with no more items than blocks has no further items)
        int next_t0 = A.total_items;
        if (t == 0 && A.total_items > (int)gridDim.x) next_t0 = (int)(gridDim.x + atomicAdd(A.work, 1u));
        const ItemPos P = item_pos<TY>(A, item);
        const int k = P.k;
        const StepInst &I = A.inst[k];
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
        // the instance's step count: the seed of the BF16 stochastic rounding
        const unsigned seed = step_seed<Store<T>::sround>(A, I, k, item, t);

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
        // this thread's halo cells: in-plane offsets, ring indices, region
        // coordinates and whether they lie inside the domain (inside the
        // region copy) rather than across a periodic seam
        u32 h_ofs[MH];
        int h_idx[MH], h_gx[MH], h_gy[MH];
        bool h_on[MH], h_dom[MH];
#pragma unroll
        for (int r = 0; r < MH; ++r) {
            int gx, gy;
            ring2_coord<TY>(min(t + r * NT, Gm::NRING2 - 1), gx, gy);
            h_ofs[r] = s_rows[gy] + s_cols[gx];
            h_idx[r] = gy * RX + gx;
            h_gx[r] = gx;
            h_gy[r] = gy;
            const int xg = x0 + gx, yg = y0 + gy;
            h_dom[r] = xg >= 0 && xg < Lx && yg >= 0 && yg < Ly;
            // a halo cell more than two cells past the upper x or y edge of
            // the lattice (in a tile the edge cuts) is read by no valid cell:
            // every stencil of the step reaches two cells.  It is neither
            // loaded nor stored; its ring slots keep values only cells whose
            // results are discarded read
            h_on[r] = ((r + 1) * NT <= Gm::NRING2 || t + r * NT < Gm::NRING2) && xg < Lx + 2 && yg < Ly + 2;
        }

        // this thread has a halo cell staged in the region copy
        const bool staged_halo = St::REGION && tma && h_on[0] && h_dom[0];
        float FA[3], FB[3], uo[3], rAo = 1.f, rBo = 0.f;
        float cprev[6];   // second-order advection: own C of plane r - 2 (see stage_u_cell)

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

            // staging buffer of this plane
            const T *stage = reinterpret_cast<const T *>(stage0);
            const float *stage_c = reinterpret_cast<const float *>(stage0 + St::C_OFF);
            // ---------------- stage M(p): radius-2 region of plane clamp(p)
            {
                const u32 pl = (u32)(min(max(p, 0), Lz - 1) * LxLy);
                MCell mh[MH];
                if (St::REGION) {
                    // halo cells across the periodic seams (not in the copied
                    // box) load first; their latency overlaps the staged work
#pragma unroll
                    for (int rr = 0; rr < MH; ++rr)
                        if (h_on[rr] && !(tma && h_dom[rr])) m_load<T>(I, fin, Cin, S, pl + h_ofs[rr], mh[rr]);
                } else {
#pragma unroll
                    for (int rr = 0; rr < MH; ++rr)
                        if (h_on[rr]) {
                            m_load<T>(I, fin, Cin, S, pl + h_ofs[rr], mh[rr]);
                            m_store<TY>(I, mh[rr], h_idx[rr], L.r3[2], ring2(p), L.cf[2]);
                        }
                }
                if (tma) {
                    if (!expired && !mbar_wait(bar, parity)) expired = true;
                    parity ^= 1u;
                }
                // early issue: the staged halo cell is read first, so that every
                // thread is done with the staging buffer after its own cell
                if (kEarlyIssue && St::REGION && staged_halo)
                    m_load_region<T, TY>(I, stage, stage_c, h_gx[0], h_gy[0], pl + h_ofs[0], mh[0]);
                {
                    // own cell; its populations wait in TMEM for stage X(p)
                    MCell m;
                    if (tma && valid) {
                        if (St::REGION)
                            m_load_region<T, TY>(I, stage, stage_c, tx + 2, ty + 2, pl + ofs_in, m);
                        else
                            m_load_staged<T, NT>(I, stage, t, Cin, S, pl + ofs_in, m);
                    } else {
                        m_load<T>(I, fin, Cin, S, pl + ofs_in, m);
                    }
                    // done with the staging buffer (early issue reads the staged
                    // halo cell before the own cell)
                    if (kEarlyIssue) mbar_arrive(ebar);
                    if constexpr (ADV2) {
                        if (p == z0 - 2)
                            for (int q6 = 0; q6 < 6; ++q6) cprev[q6] = m.c[q6];
                    }
                    m_store<TY>(I, m, idx_in, L.r3[2], ring2(p), L.cf[2]);
                    tm_store38(tm_warp + (u32)((p & 1) * 64), reinterpret_cast<const float *>(m.ab));
                }
                if (St::REGION) {
#pragma unroll
                    for (int rr = 0; rr < MH; ++rr)
                        if (h_on[rr]) {
                            if (!kEarlyIssue && tma && h_dom[rr])
                                m_load_region<T, TY>(I, stage, stage_c, h_gx[rr], h_gy[rr], pl + h_ofs[rr], mh[rr]);
                            m_store<TY>(I, mh[rr], h_idx[rr], L.r3[2], ring2(p), L.cf[2]);
                        }
                }
            }
            // the staging buffer is free once every thread has read its cells:
            // start the copy of the next plane (of this item, else the first
            // plane of the block's next item); with early issue before the
            // stage-M barrier, while the others still compute their halo cells
            auto issue_next = [&]() {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                const u32 go = expired ? 0u : 1u;
                if (p + 1 <= z1 + 1) {
                    if (tma) {
                        issue_plane<T, TY>(A, P, p + 1, stage_addr, bar, go);
                        issued += go;
                    }
                } else {
                    const int nx = s_item[slot ^ 1];   // published at the item's first plane
                    if (nx < A.total_items) {
                        const ItemPos Pn = item_pos<TY>(A, nx);
                        if (A.inst[Pn.k].tma) {
                            issue_plane<T, TY>(A, Pn, Pn.z0 - 2, stage_addr, bar, go);
                            issued += go;
                        }
                    }
                }
            };
            if (kEarlyIssue && t == kIssuer) {
                if (!expired && !mbar_wait(ebar, eparity)) expired = true;
                eparity ^= 1u;
                issue_next();
            }
            __syncthreads();
            if (t == 0 && p == z0 - 2) s_item[slot ^ 1] = next_t0;
            if (!kEarlyIssue && t == 0) issue_next();
            // the collision's populations start to come back from TMEM here (or
            // just before the collision) and are waited for after stage F
            const bool doX = q >= z0 && q < z1;
            u32 tr[38];
            if (kEarlyTmem && doX) {
                const u32 ta = tm_warp + (u32)((q & 1) * 64);
                tm_wait_st();
                tm_ld32(ta, tr);
                tm_ld4(ta + 32, tr + 32);
                tm_ld2(ta + 36, tr + 36);
            }
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
            if (doX) {
                if (!kEarlyTmem) {
                    const u32 ta = tm_warp + (u32)((q & 1) * 64);
                    tm_wait_st();
                    tm_ld32(ta, tr);
                    tm_ld4(ta + 32, tr + 32);
                    tm_ld2(ta + 36, tr + 36);
                }
                tm_wait_ld38(tr);
                float2 fx[Q];
#pragma unroll
                for (int i = 0; i < Q; ++i) fx[i] = make_float2(__uint_as_float(tr[2 * i]), __uint_as_float(tr[2 * i + 1]));
                if (valid) {
                    const u32 nq = (u32)(q * LxLy) + ofs_in;
                    const float rt = rAo + rBo;
                    if (!(rt > 0.f) || uo[0] != uo[0] || uo[1] != uo[1] || uo[2] != uo[2])
                        raise_step_flag(A.status, I, kFlagDiverged);
                    // omega = 1 / (3 nu + 1/2), nu = (rho_A nu_A + rho_B nu_B) / rho
                    const float om = rt / (3.0f * (rAo * I.nu_A + rBo * I.nu_B) + 0.5f * rt);
                    const bool bottom = q == 0, top = q == Lz - 1;
                    PushOffsets Po;
                    const float2 *rho_s = reinterpret_cast<const float2 *>(smem() + Rg::RHO);
                    Po.ring[0] = rho_s + L.r3[0] * R2N;
                    Po.ring[1] = rho_s + L.r3[1] * R2N;
                    Po.ring[2] = rho_s + L.r3[2] * R2N;
                    Po.idx = idx_in;
                    Po.own = make_float2(rAo, rBo);
                    Po.track = I.dens_out != nullptr;
                    Po.r0 = make_float2(I.rho0A, I.rho0B);
                    Po.seed = seed;
                    const float2 F2[3] = {make_float2(FA[0], FB[0]), make_float2(FA[1], FB[1]),
                                          make_float2(FA[2], FB[2])};
                    if (!kSplitWalls || bottom || top)
                        collide_push_ab<T, true, RX>(fx, fout, S, Po.own, Po, uo, F2, om, nq, bottom, top, Uw, LxLy,
                                                     dxy);
                    else
                        collide_push_ab<T, false, RX>(fx, fout, S, Po.own, Po, uo, F2, om, nq, false, false, Uw,
                                                      LxLy, dxy);
                    // this step's densities: the offsets of the state just written
                    if (Store<T>::offset && Po.track) I.dens_out[nq] = Po.own;
                }
            }
            // ---------------- stage U(r): FENE-P update, Eq. 2 (Eq. 4).  It
            // reads u of plane r on the radius-1 region (complete since the
            // previous plane's barriers) and u of plane q of its own cell only
            // (written above by this thread), so it needs no barrier after
            // stage F: threads without halo work in stage F go on to it.
            if (r >= z0 && r < z1 && valid) {
                float cn[6];
                if (!stage_u_cell<TY, ADV2>(I, idx_in, L, r, cn, cprev)) raise_step_flag(A.status, I, kFlagDiverged);
                const u32 n = (u32)(r * LxLy) + ofs_in;
#pragma unroll
                for (int q6 = 0; q6 < 6; ++q6) Cout[(u32)(q6 * S + n)] = cn[q6];
            }
            __syncthreads();  // stages F, X and U done with the rings before stage M(p+1)
        }
        item = s_item[slot ^ 1];   // published in the first iteration, several barriers ago
        slot ^= 1;
    }

    if (t == 0 && A.total_items > (int)gridDim.x) release_work_counters(A.work);
    if (expired) {
        // issuer: the copy whose wait expired may still be in flight (no
        // later one was issued); wait for its phase once more, bounded,
        // before the block's shared memory is released
        if (t == kIssuer && issued > 0) mbar_wait(bar, (issued - 1u) & 1u);
        atomicOr(A.status, kFlagTimeout);
    }
    tm_wait_st();   // no TMEM store may be pending when the columns are freed
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    if (ty == 0) tm_dealloc(s_tmem, Gm::TMEM_COLS);
}

// ---------------------------------------------------------------- host side
namespace {

void fill_inst(StepInst &d, const InstDev &I, const PopMaps *maps, const StepMaps *maps_dev, int cur) {
    d = StepInst{};
    if (maps && maps->ok && maps_dev) {
        d.maps = maps_dev + cur;
        d.tma = 1;
    }
    d.Lx = (unsigned short)I.Lx;
    d.Ly = (unsigned short)I.Ly;
    d.Lz = (unsigned short)I.Lz;
    d.LxLy = (u32)(I.Lx * I.Ly);
    d.visc_comp = (signed char)I.visc_comp;
    d.ntx = (unsigned short)I.ntx;
    d.nty = (unsigned short)I.nty;
    d.zc = (unsigned short)I.zc;
    d.S = (u32)I.S;
    d.fin = I.f[cur];
    d.fout = I.f[cur ^ 1];
    d.Cin = I.C[cur];
    d.Cout = I.C[cur ^ 1];
    d.dens_in = I.dens[cur ^ 1];
    d.dens_out = I.dens[cur];
    d.status = I.status;
    d.step_ctr = I.step_ctr;
    d.parity = (unsigned char)cur;
    d.G = I.G;
    d.Uw = I.Uw;
    d.nu_A = I.nu_A;
    d.nu_B = I.nu_B;
    d.pi_coef = I.pi_coef;
    d.L2 = I.L2;
    d.inv_tauP = I.inv_tauP;
    d.gx = I.gx;
    d.gy = I.gy;
    d.gz = I.gz;
    d.rho0A = I.rho0[0];
    d.rho0B = I.rho0[1];
}

// Dynamic shared memory: rings, alignment slack, TMA staging buffer.
template <typename T, int TY>
constexpr size_t smem_bytes() {
    return sizeof(float) * Geom<TY>::FLOATS + 128 + Stage<T, TY>::BYTES;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

template <typename T, int TY, bool ADV2>
cudaError_t cell_launch_t(const StepArgs &a, int grid, cudaStream_t st) {
    k_fused<T, TY, ADV2><<<grid, Geom<TY>::NT, smem_bytes<T, TY>(), st>>>(a);
    return cudaGetLastError();
}

template <int TY, bool ADV2 = false>
cudaError_t cell_launch_ty(const StepArgs &a, int grid, int precision, cudaStream_t st) {
    switch (precision) {
        case LBFE_FP16_OFFSET: return cell_launch_t<__half, TY, ADV2>(a, grid, st);
        case LBFE_BF16_OFFSET: return cell_launch_t<__nv_bfloat16, TY, ADV2>(a, grid, st);
        default: return cell_launch_t<float, TY, ADV2>(a, grid, st);
    }
}

template <typename T, int TY, bool ADV2>
cudaError_t prep_t(int *bps) {
    const size_t smem = smem_bytes<T, TY>();
    cudaError_t e =
        cudaFuncSetAttribute(k_fused<T, TY, ADV2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int b = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_fused<T, TY, ADV2>, Geom<TY>::NT, smem);
    if (e != cudaSuccess) return e;
    // resident blocks of one SM share its 512 TMEM columns
    const int tm = 512 / Geom<TY>::TMEM_COLS;
    *bps = b < tm ? b : tm;
    return cudaSuccess;
}

template <int TY, bool ADV2 = false>
cudaError_t prep_ty(int precision, int *bps) {
    switch (precision) {
        case LBFE_FP16_OFFSET: return prep_t<__half, TY, ADV2>(bps);
        case LBFE_BF16_OFFSET: return prep_t<__nv_bfloat16, TY, ADV2>(bps);
        default: return prep_t<float, TY, ADV2>(bps);
    }
}

// One launch over instances [k0, k1) (at most kStepMaxInst of them).
cudaError_t fused_group(const LaunchCtx &c, int cur, int k0, int k1) {
    StepArgs a{};
    a.n = k1 - k0;
    a.status = c.status;
    a.work = c.status + 2;
    const int base = c.item_off_host[k0];
    for (int k = k0; k < k1; ++k) {
        a.item_off[k - k0] = c.item_off_host[k] - base;
        fill_inst(a.inst[k - k0], c.inst_host[k], c.maps_host ? c.maps_host + k : nullptr,
                  c.maps_dev ? c.maps_dev + 2 * k : nullptr, cur);
    }
    a.item_off[a.n] = c.item_off_host[k1] - base;
    a.total_items = a.item_off[a.n];
    if (a.total_items <= 0) return cudaSuccess;
    const int grid = a.total_items < c.fused_slots ? a.total_items : c.fused_slots;
    if (c.step_kernel == LBFE_STEP_PAIR) return step_pair_launch(a, grid, c.precision, c.stream);
    return step_cell_launch(a, grid, c.tile_y, c.precision, c.advection, c.stream);
}

}  // namespace

cudaError_t step_cell_launch(const StepArgs &a, int grid, int tile_y, int precision, int advection,
                             cudaStream_t st) {
    // the second-order advection scheme runs at 8-row tiles only
    if (advection == 1) return cell_launch_ty<8, true>(a, grid, precision, st);
    switch (tile_y) {
        case 12: return cell_launch_ty<12>(a, grid, precision, st);
        case 16: return cell_launch_ty<16>(a, grid, precision, st);
        default: return cell_launch_ty<8>(a, grid, precision, st);
    }
}

cudaError_t step_cell_prepare(int tile_y, int precision, int advection, int *blocks_per_sm) {
    if (advection == 1) return prep_ty<8, true>(precision, blocks_per_sm);
    switch (tile_y) {
        case 12: return prep_ty<12>(precision, blocks_per_sm);
        case 16: return prep_ty<16>(precision, blocks_per_sm);
        default: return prep_ty<8>(precision, blocks_per_sm);
    }
}

cudaError_t launch_fused(const LaunchCtx &c, int cur) {
    for (int k0 = 0; k0 < c.n; k0 += kStepMaxInst) {
        const int k1 = k0 + kStepMaxInst < c.n ? k0 + kStepMaxInst : c.n;
        cudaError_t e = fused_group(c, cur, k0, k1);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int fused_launches(int n) { return n <= 1 ? 1 : (n + kStepMaxInst - 1) / kStepMaxInst; }

// The populations of an instance viewed as a 4-D tensor (x, y, z, s*19 + i)
// with strides (1, Lx, Lx Ly, S) elements, the conformation as
// (x, y, z, component) and the offset densities as (x, y, z) of 8-byte
// float2; boxes as in Stage.  TMA needs every stride to be a multiple of
// 16 bytes, so instances with Lx * element size not divisible by 16 keep
// ordinary loads.
cudaError_t fused_pop_maps(const InstDev &I, int precision, int tile_y, bool short_box, PopMaps *m) {
    std::memset(m, 0, sizeof *m);
    const size_t esz = precision == LBFE_FP32 ? 4 : 2;
    if (((size_t)I.Lx * esz) % 16 != 0 || ((size_t)I.Lx * 4) % 16 != 0) return cudaSuccess;
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return cudaSuccess;
    const CUtensorMapDataType dt = precision == LBFE_FP16_OFFSET   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                   : precision == LBFE_BF16_OFFSET ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                                   : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const bool region = tile_y <= 12;
    const cuuint32_t xpad = (cuuint32_t)(16 / esz), ty = (cuuint32_t)tile_y;
    const cuuint64_t dims[4] = {(cuuint64_t)I.Lx, (cuuint64_t)I.Ly, (cuuint64_t)I.Lz, (cuuint64_t)(2 * Q)};
    const cuuint64_t strides[3] = {(cuuint64_t)I.Lx * esz, (cuuint64_t)I.Lx * I.Ly * esz, (cuuint64_t)I.S * esz};
    const cuuint32_t box[4] = {region ? 32u + 2 * xpad : 32u, (region ? ty + 4 : ty) - (short_box ? 1u : 0u), 1u,
                               (cuuint32_t)(2 * Q)};
    const cuuint64_t cdims[4] = {(cuuint64_t)I.Lx, (cuuint64_t)I.Ly, (cuuint64_t)I.Lz, 6};
    const cuuint64_t cstrides[3] = {(cuuint64_t)I.Lx * 4, (cuuint64_t)I.Lx * I.Ly * 4, (cuuint64_t)I.S * 4};
    const cuuint32_t cbox[4] = {40u, ty + 4, 1u, 6u};
    const cuuint64_t ddims[3] = {(cuuint64_t)I.Lx, (cuuint64_t)I.Ly, (cuuint64_t)I.Lz};
    const cuuint64_t dstrides[2] = {(cuuint64_t)I.Lx * 8, (cuuint64_t)I.Lx * I.Ly * 8};
    const cuuint32_t dbox[3] = {36u, ty + 4, 1u};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    auto enc = [&](CUtensorMap *map, CUtensorMapDataType t, cuuint32_t rank, void *base, const cuuint64_t *d,
                   const cuuint64_t *st, const cuuint32_t *bx) {
        return fn(map, t, rank, base, d, st, bx, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    };
    for (int b = 0; b < 2; ++b) {
        StepMaps &sm = m->m[b];
        CUresult r = enc(&sm.pop, dt, 4, I.f[b], dims, strides, box);
        if (r == CUDA_SUCCESS && region)
            r = enc(&sm.c, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, I.C[b], cdims, cstrides, cbox);
        // the state in f[b] is stored relative to dens[b ^ 1]
        if (r == CUDA_SUCCESS && region && esz == 2 && I.dens[b ^ 1])
            r = enc(&sm.dens, CU_TENSOR_MAP_DATA_TYPE_INT64, 3, I.dens[b ^ 1], ddims, dstrides, dbox);
        if (r != CUDA_SUCCESS) {
            std::memset(m, 0, sizeof *m);
            return cudaSuccess;
        }
    }
    m->ok = 1;
    return cudaSuccess;
}

cudaError_t fused_prepare(int step_kernel, int tile_y, int precision, int advection, int *blocks_per_sm) {
    if (step_kernel == LBFE_STEP_PAIR) return step_pair_prepare(precision, blocks_per_sm);
    return step_cell_prepare(tile_y, precision, advection, blocks_per_sm);
}

}  // namespace lbfe
