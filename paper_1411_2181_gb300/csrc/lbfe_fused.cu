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
    static constexpr int NHALO = R2N - NT;             // radius-2 cells outside the tile
    static constexpr int NRING1 = 2 * (RX - 2) + 2 * TY;  // radius-1 cells outside the tile
    // rings: rho (float2) x3, Pi 6x3, j 3x2, C 6x4, u 3x3
    static constexpr int FLOATS = (2 * 3 + 18 + 6 + 24 + 9) * R2N;
};

__device__ __forceinline__ int ring3(int p) { return (p + 12) % 3; }
__device__ __forceinline__ int ring4(int p) { return (p + 12) & 3; }
__device__ __forceinline__ int ring2(int p) { return (p + 12) & 1; }
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

// Halo cell h (0 <= h < NHALO) of the radius-2 region: two rows below and
// above the tile (full width), then two columns left and right of it.
template <int TY>
__device__ __forceinline__ void halo2_coord(int h, int &gx, int &gy) {
    using Gm = Geom<TY>;
    if (h < 4 * Gm::RX) {
        const int rr = h / Gm::RX;
        gx = h - rr * Gm::RX;
        gy = rr < 2 ? rr : Gm::RY - 4 + rr;
    } else {
        const int h2 = h - 4 * Gm::RX;
        const int cc = h2 / TY;
        gy = 2 + (h2 - cc * TY);
        gx = cc < 2 ? cc : Gm::RX - 4 + cc;
    }
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

struct Rings {
    float2 *rho;   // [3][R2N]
    float *pi;     // [3][6][R2N]
    float *j;      // [2][3][R2N]
    float *c;      // [4][6][R2N]
    float *u;      // [3][3][R2N]
};

// Stage M for one cell: moments, stress and conformation into the rings.
template <typename T, int TY>
__device__ __forceinline__ void stage_m_cell(const InstDev &I, const T *__restrict__ fin,
                                             const float *__restrict__ Cin, long long n, int idx,
                                             const Rings &R, int p) {
    constexpr int R2N = Geom<TY>::R2N;
    const long long S = I.S;
    const float ra0 = I.rho0[0], rb0 = I.rho0[1];
    float fa[Q], fb[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        fa[i] = ldpop(fin + (long long)i * S + n, wq(i) * ra0);
        fb[i] = ldpop(fin + (long long)(Q + i) * S + n, wq(i) * rb0);
    }
    float c[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) c[k] = __ldg(Cin + (long long)k * S + n);
    float rA = 0.f, rB = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) { rA += fa[i]; rB += fb[i]; }
    // momentum from opposite-pair differences (exact in FP32 per pair)
    float jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const float d = (fa[i] - fa[i + 1]) + (fb[i] - fb[i + 1]);
        if (cx(i)) jx += cx(i) * d;
        if (cy(i)) jy += cy(i) * d;
        if (cz(i)) jz += cz(i) * d;
    }
    const int s3 = ring3(p), s2 = ring2(p), s4 = ring4(p);
    R.rho[s3 * R2N + idx] = make_float2(rA, rB);
    float *jr = R.j + s2 * 3 * R2N;
    jr[idx] = jx;
    jr[R2N + idx] = jy;
    jr[2 * R2N + idx] = jz;
    float *cr = R.c + s4 * 6 * R2N;
#pragma unroll
    for (int k = 0; k < 6; ++k) cr[k * R2N + idx] = c[k];
    float a = 0.f, fp = 1.f;
    if (I.visc_comp >= 0) {
        a = I.pi_coef * (I.visc_comp == 0 ? rA : rB) / (rA + rB);
        fp = peterlin(I.L2, c[0], c[1], c[2]);
    }
    float *pr = R.pi + s3 * 6 * R2N;
#pragma unroll
    for (int k = 0; k < 6; ++k) pr[k * R2N + idx] = a * (fp * c[k] - (k < 3 ? 1.f : 0.f));
}

// Stage F for one cell of plane q: forces and velocity.  Writes u to the
// ring; returns the per-component total forces, u and the densities.
template <int TY>
__device__ __forceinline__ void stage_f_cell(const InstDev &I, int idx, const Rings &R, int q,
                                             float FA[3], float FB[3], float u[3], float &rA, float &rB) {
    constexpr int R2N = Geom<TY>::R2N, RX = Geom<TY>::RX;
    const float2 *rm = R.rho + ring3(q - 1) * R2N;
    const float2 *rc = R.rho + ring3(q) * R2N;
    const float2 *rp = R.rho + ring3(q + 1) * R2N;
    const float2 r0 = rc[idx];
    rA = r0.x;
    rB = r0.y;
    // Shan-Chen with opposite neighbours in pairs
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
    // polymer force F_P,a = sum_b (Pi_ba(x + e_b) - Pi_ba(x - e_b))/2
    float FP[3] = {0.f, 0.f, 0.f};
    if (I.visc_comp >= 0) {
        const float *pm = R.pi + ring3(q - 1) * 6 * R2N;
        const float *pc = R.pi + ring3(q) * 6 * R2N;
        const float *pp = R.pi + ring3(q + 1) * 6 * R2N;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float gxd = pc[symk(0, a) * R2N + idx + 1] - pc[symk(0, a) * R2N + idx - 1];
            const float gyd = pc[symk(1, a) * R2N + idx + RX] - pc[symk(1, a) * R2N + idx - RX];
            const float gzd = pp[symk(2, a) * R2N + idx] - pm[symk(2, a) * R2N + idx];
            FP[a] = 0.5f * (gxd + gyd + gzd);
        }
    }
    const float *jr = R.j + ring2(q) * 3 * R2N;
    const float g[3] = {I.gx, I.gy, I.gz};
    const float inv = 1.0f / (rA + rB);
    float *ur = R.u + ring3(q) * 3 * R2N;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        FA[a] = -I.G * rA * sA[a] + (rA * inv) * FP[a] + rA * g[a];
        FB[a] = -I.G * rB * sB[a] + (rB * inv) * FP[a] + rB * g[a];
        u[a] = (jr[a * R2N + idx] + 0.5f * (FA[a] + FB[a])) * inv;
        ur[a * R2N + idx] = u[a];
    }
}

}  // namespace

template <typename T, int TY>
__global__ void __launch_bounds__(32 * TY, TY >= 16 ? 1 : (TY >= 8 ? 2 : 3))
k_fused(const InstDev *__restrict__ insts, const int *__restrict__ item_off, int n_inst, int total_items,
        int cur, unsigned *status) {
    using Gm = Geom<TY>;
    constexpr int TX = Gm::TX, NT = Gm::NT, RX = Gm::RX, R2N = Gm::R2N;
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    Rings R;
    R.rho = reinterpret_cast<float2 *>(sm);
    R.pi = sm + 6 * R2N;
    R.j = R.pi + 18 * R2N;
    R.c = R.j + 6 * R2N;
    R.u = R.c + 24 * R2N;

    const int t = threadIdx.x, tx = t & 31, ty = t >> 5;
    const int gxi = tx + 2, gyi = ty + 2, idx_in = gyi * RX + gxi;

    for (int item = blockIdx.x; item < total_items; item += gridDim.x) {
        const int k = find_inst(item_off, n_inst, item);
        const InstDev &I = insts[k];
        const int Lx = I.Lx, Ly = I.Ly, Lz = I.Lz;
        const long long LxLy = (long long)Lx * Ly, S = I.S;
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

        // own cell and its periodic neighbours
        const int x = bx * TX + tx, y = by * TY + ty;
        const bool valid = x < Lx && y < Ly;
        const long long ofs_in = (long long)wrapg(y, Ly) * Lx + wrapg(x, Lx);
        const int xm = wrapg(x - 1, Lx), xp = wrapg(x + 1, Lx);
        const long long rowm = (long long)wrapg(y - 1, Ly) * Lx, row0 = (long long)wrapg(y, Ly) * Lx,
                        rowp = (long long)wrapg(y + 1, Ly) * Lx;
        const int xw = wrapg(x, Lx);

        float FA[3], FB[3], uo[3], rAo = 1.f, rBo = 0.f;

        for (int p = z0 - 2; p <= z1 + 1; ++p) {
            // ---------------- stage M(p): radius-2 region of plane clamp(p)
            {
                const long long pl = (long long)min(max(p, 0), Lz - 1) * LxLy;
                stage_m_cell<T, TY>(I, fin, Cin, pl + ofs_in, idx_in, R, p);
                for (int h = t; h < Gm::NHALO; h += NT) {
                    int gx, gy;
                    halo2_coord<TY>(h, gx, gy);
                    const long long o = (long long)wrapg(y0 + gy, Ly) * Lx + wrapg(x0 + gx, Lx);
                    stage_m_cell<T, TY>(I, fin, Cin, pl + o, gy * RX + gx, R, p);
                }
            }
            __syncthreads();
            // ---------------- stage F(q): radius-1 region
            const int q = p - 1;
            const bool doF = q >= max(z0 - 1, 0) && q <= min(z1, Lz - 1);
            if (doF) {
                stage_f_cell<TY>(I, idx_in, R, q, FA, FB, uo, rAo, rBo);
                for (int h = t; h < Gm::NRING1; h += NT) {
                    int gx, gy;
                    ring1_coord<TY>(h, gx, gy);
                    float a[3], b[3], uu[3], ra, rb;
                    stage_f_cell<TY>(I, gy * RX + gx, R, q, a, b, uu, ra, rb);
                }
            }
            __syncthreads();
            // ---------------- stage X(q): collision + push streaming
            if (q >= z0 && q < z1 && valid) {
                const float rt = rAo + rBo;
                if (!(rt > 0.f) || uo[0] != uo[0] || uo[1] != uo[1] || uo[2] != uo[2])
                    atomicOr(status, kFlagDiverged);
                const float nu = (rAo * I.nu_A + rBo * I.nu_B) / rt;
                const float om = 1.0f / (3.0f * nu + 0.5f);
                const float pref = 1.0f - 0.5f * om;
                const float uu = uo[0] * uo[0] + uo[1] * uo[1] + uo[2] * uo[2];
                const long long n = (long long)q * LxLy + ofs_in;
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const float rs = s == 0 ? rAo : rBo;
                    const float r0s = I.rho0[s];
                    const float Fx = s == 0 ? FA[0] : FB[0], Fy = s == 0 ? FA[1] : FB[1],
                                Fz = s == 0 ? FA[2] : FB[2];
                    const float uF = uo[0] * Fx + uo[1] * Fy + uo[2] * Fz;
                    float fv[Q];
#pragma unroll
                    for (int i = 0; i < Q; ++i) fv[i] = ldpop(fin + (long long)(s * Q + i) * S + n, wq(i) * r0s);
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        const float cu = cx(i) * uo[0] + cy(i) * uo[1] + cz(i) * uo[2];
                        const float cF = cx(i) * Fx + cy(i) * Fy + cz(i) * Fz;
                        const float feq = wq(i) * rs * (1.f + 3.f * cu + 4.5f * cu * cu - 1.5f * uu);
                        const float src = pref * wq(i) * (3.f * (cF - uF) + 9.f * cu * cF);
                        float v = fv[i] - om * (fv[i] - feq) + src;
                        const int zd = q + cz(i);
                        int dir = i;
                        long long dst;
                        if (zd < 0 || zd >= Lz) {
                            // halfway bounce-back, moving-wall term -6 w_i rho_s (c_i . U_wall)
                            const float uw = zd < 0 ? -I.Uw : I.Uw;
                            v -= 6.f * wq(i) * rs * (float)cx(i) * uw;
                            dir = opp(i);
                            dst = n;
                        } else {
                            const long long row = cy(i) > 0 ? rowp : (cy(i) < 0 ? rowm : row0);
                            const int col = cx(i) > 0 ? xp : (cx(i) < 0 ? xm : xw);
                            dst = (long long)zd * LxLy + row + col;
                        }
                        if (Store<T>::offset) v -= wq(i) * r0s;
                        Store<T>::st(fout + (long long)(s * Q + dir) * S + dst, v);
                    }
                }
            }
            // ---------------- stage U(r): FENE-P update
            const int r = p - 2;
            if (r >= z0 && r < z1 && valid) {
                const float *um = R.u + ring3(r - 1) * 3 * R2N;
                const float *uc = R.u + ring3(r) * 3 * R2N;
                const float *up = R.u + ring3(r + 1) * 3 * R2N;
                const float *cm = R.c + ring4(r - 1) * 6 * R2N;
                const float *cc = R.c + ring4(r) * 6 * R2N;
                const float *cp = R.c + ring4(r + 1) * 6 * R2N;
                const int i0 = idx_in;
                float u0[3], Gr[3][3];
#pragma unroll
                for (int j = 0; j < 3; ++j) u0[j] = uc[j * R2N + i0];
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const float uwb = j == 0 ? -I.Uw : 0.f, uwt = j == 0 ? I.Uw : 0.f;
                    const float uzp = (r == Lz - 1) ? 2.f * uwt - u0[j] : up[j * R2N + i0];
                    const float uzm = (r == 0) ? 2.f * uwb - u0[j] : um[j * R2N + i0];
                    Gr[0][j] = 0.5f * (uc[j * R2N + i0 + 1] - uc[j * R2N + i0 - 1]);
                    Gr[1][j] = 0.5f * (uc[j * R2N + i0 + RX] - uc[j * R2N + i0 - RX]);
                    Gr[2][j] = 0.5f * (uzp - uzm);
                }
                float c[6];
#pragma unroll
                for (int q6 = 0; q6 < 6; ++q6) c[q6] = cc[q6 * R2N + i0];
                float adv[6];
#pragma unroll
                for (int q6 = 0; q6 < 6; ++q6) {
                    const float *col = cc + q6 * R2N;
                    const float ax = u0[0] > 0.f ? (c[q6] - col[i0 - 1]) : (col[i0 + 1] - c[q6]);
                    const float ay = u0[1] > 0.f ? (c[q6] - col[i0 - RX]) : (col[i0 + RX] - c[q6]);
                    const float az = u0[2] > 0.f ? (c[q6] - cm[q6 * R2N + i0]) : (cp[q6 * R2N + i0] - c[q6]);
                    adv[q6] = u0[0] * ax + u0[1] * ay + u0[2] * az;
                }
                const float Cm[3][3] = {{c[0], c[3], c[4]}, {c[3], c[1], c[5]}, {c[4], c[5], c[2]}};
                const float fp = peterlin(I.L2, c[0], c[1], c[2]);
                const long long n = (long long)r * LxLy + ofs_in;
#pragma unroll
                for (int q6 = 0; q6 < 6; ++q6) {
                    const int a = q6 < 3 ? q6 : (q6 == 5 ? 1 : 0);
                    const int b = q6 < 3 ? q6 : (q6 == 3 ? 1 : 2);
                    float st = 0.f;
#pragma unroll
                    for (int m = 0; m < 3; ++m) st += Cm[a][m] * Gr[m][b] + Gr[m][a] * Cm[m][b];
                    const float relax = (fp * c[q6] - (q6 < 3 ? 1.f : 0.f)) * I.inv_tauP;
                    Cout[(long long)q6 * S + n] = c[q6] + (-adv[q6] + st - relax);
                }
                if (!(c[0] + c[1] + c[2] < I.L2)) atomicOr(status, kFlagDiverged);
            }
            __syncthreads();
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
