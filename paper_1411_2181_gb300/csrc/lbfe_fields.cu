// lbfe_fields.cu -- field queries and state set-up, one thread per cell:
//   moments  rho_A, rho_B and the total momentum j of the streamed
//            populations (the densities the caller asks for);
//   forces   Shan-Chen force, polymer-stress divergence (Eqs. 1 and 3, last
//            term) and the Guo velocity u = (j + F/2)/rho (the velocity
//            field the caller asks for);
//   init     f = f^eq(rho_s, 0), C = I;
//   decode / encode of one population array for host copies.
// The time step itself is the fused kernel (lbfe_fused.cu).  Every instance
// of a batch is covered by one launch through the tile table (tile_off).
#include "lbfe_internal.cuh"

namespace lbfe {

template <typename T>
__device__ __forceinline__ float decode(const T *f, long long off, int i, float r0) {
    float v = Store<T>::ld(f + off);
    if (Store<T>::offset) v += wq(i) * r0;
    return v;
}

#define LBFE_CELL_PROLOGUE                                                                  \
    const int k = find_inst(tile_off, n_inst, blockIdx.x);                                  \
    const InstDev &I = insts[k];                                                            \
    const long long n = (long long)(blockIdx.x - __ldg(tile_off + k)) * kBlock + threadIdx.x; \
    if (n >= I.N) return;                                                                   \
    const long long S = I.S;                                                                \
    const int Lx = I.Lx, Ly = I.Ly, Lz = I.Lz;                                              \
    const int x = (int)(n % Lx);                                                            \
    const int y = (int)((n / Lx) % Ly);                                                     \
    const int z = (int)(n / ((long long)Lx * Ly));                                          \
    (void)x; (void)y; (void)z; (void)Lz;

// ---------------------------------------------------------------- pass 1
template <typename T>
__global__ void __launch_bounds__(kBlock)
k_moments(const InstDev *__restrict__ insts, const int *__restrict__ tile_off, int n_inst, int cur) {
    LBFE_CELL_PROLOGUE
    const T *f = (const T *)I.f[cur];
    const float2 od = offset_dens<T>(I, cur, n);
    // momentum from opposite-pair differences f_i - f_opp(i): the pair
    // members are close, so each difference is exact in FP32 and the large
    // cancellation of the plain signed sum is avoided
    float r[2], jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const float r0 = s == 0 ? od.x : od.y;
        float v[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) v[i] = decode(f, (long long)(s * Q + i) * S + n, i, r0);
        float acc = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) acc += v[i];
#pragma unroll
        for (int i = 1; i < Q; i += 2) {
            const float d = v[i] - v[i + 1];
            if (cx(i)) jx += cx(i) * d;
            if (cy(i)) jy += cy(i) * d;
            if (cz(i)) jz += cz(i) * d;
        }
        r[s] = acc;
    }
    I.rho[n] = r[0];
    I.rho[S + n] = r[1];
    I.jm[n] = jx;
    I.jm[S + n] = jy;
    I.jm[2 * S + n] = jz;
}

// Row b of the polymer stress Pi at cell m: (Pi_bx, Pi_by, Pi_bz).
__device__ __forceinline__ void stress_row(const InstDev &I, const float *__restrict__ C,
                                           long long m, int b, float out[3]) {
    const long long S = I.S;
    const float *__restrict__ rho = I.rho;
    const float rA = __ldg(rho + m), rB = __ldg(rho + S + m);
    const float chi = (I.visc_comp == 0 ? rA : rB) / (rA + rB);
    const float c0 = __ldg(C + m), c1 = __ldg(C + S + m), c2 = __ldg(C + 2 * S + m);
    const float fp = peterlin(I.L2, c0, c1, c2);
    const float a = I.pi_coef * chi;
    float r0, r1, r2;  // C row b
    if (b == 0) { r0 = c0; r1 = __ldg(C + 3 * S + m); r2 = __ldg(C + 4 * S + m); }
    else if (b == 1) { r0 = __ldg(C + 3 * S + m); r1 = c1; r2 = __ldg(C + 5 * S + m); }
    else { r0 = __ldg(C + 4 * S + m); r1 = __ldg(C + 5 * S + m); r2 = c2; }
    out[0] = a * (fp * r0 - (b == 0 ? 1.f : 0.f));
    out[1] = a * (fp * r1 - (b == 1 ? 1.f : 0.f));
    out[2] = a * (fp * r2 - (b == 2 ? 1.f : 0.f));
}

// ---------------------------------------------------------------- pass 2
__global__ void __launch_bounds__(kBlock)
k_forces(const InstDev *__restrict__ insts, const int *__restrict__ tile_off, int n_inst, int cur) {
    LBFE_CELL_PROLOGUE
    const float *__restrict__ rho = I.rho;
    const float rA = rho[n], rB = rho[S + n], rt = rA + rB;

    // Shan-Chen: F_s = -G rho_s sum_i w_i rho_t(x + c_i) c_i, densities
    // beyond a wall taken from the adjacent layer
    float sA[3] = {0.f, 0.f, 0.f}, sB[3] = {0.f, 0.f, 0.f};
    // opposite neighbours in pairs: w_i c_i (rho(x + c_i) - rho(x - c_i))
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const long long mp = ((long long)min(max(z + cz(i), 0), Lz - 1) * Ly + wrapi(y + cy(i), Ly)) * Lx +
                             wrapi(x + cx(i), Lx);
        const long long mm = ((long long)min(max(z - cz(i), 0), Lz - 1) * Ly + wrapi(y - cy(i), Ly)) * Lx +
                             wrapi(x - cx(i), Lx);
        const float dA = __ldg(rho + mp) - __ldg(rho + mm);
        const float dB = __ldg(rho + S + mp) - __ldg(rho + S + mm);
        const float w = wq(i);
        if (cx(i)) { sA[0] += cx(i) * w * dB; sB[0] += cx(i) * w * dA; }
        if (cy(i)) { sA[1] += cy(i) * w * dB; sB[1] += cy(i) * w * dA; }
        if (cz(i)) { sA[2] += cz(i) * w * dB; sB[2] += cz(i) * w * dA; }
    }
    float FP[3] = {0.f, 0.f, 0.f};
    if (I.visc_comp >= 0) {
        // F_P,a = sum_b (Pi_ba(x + e_b) - Pi_ba(x - e_b))/2, Pi mirrored at walls
        const float *__restrict__ C = I.C[cur];
        const int xp = wrapi(x + 1, Lx), xm = wrapi(x - 1, Lx);
        const int yp = wrapi(y + 1, Ly), ym = wrapi(y - 1, Ly);
        const int zp = min(z + 1, Lz - 1), zm = max(z - 1, 0);
        const long long row = ((long long)z * Ly + y) * Lx;
        long long mp[3] = {row + xp, ((long long)z * Ly + yp) * Lx + x, ((long long)zp * Ly + y) * Lx + x};
        long long mm[3] = {row + xm, ((long long)z * Ly + ym) * Lx + x, ((long long)zm * Ly + y) * Lx + x};
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            float pp[3], pm[3];
            stress_row(I, C, mp[b], b, pp);
            stress_row(I, C, mm[b], b, pm);
            FP[0] += 0.5f * (pp[0] - pm[0]);
            FP[1] += 0.5f * (pp[1] - pm[1]);
            FP[2] += 0.5f * (pp[2] - pm[2]);
        }
    }
    const float g[3] = {I.gx, I.gy, I.gz};
    const float inv_rt = 1.0f / rt;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float fa = -I.G * rA * sA[a] + (rA * inv_rt) * FP[a] + rA * g[a];
        const float fb = -I.G * rB * sB[a] + (rB * inv_rt) * FP[a] + rB * g[a];
        I.F[a * S + n] = fa;
        I.F[(3 + a) * S + n] = fb;
        I.u[a * S + n] = (I.jm[a * S + n] + 0.5f * (fa + fb)) * inv_rt;
    }
}

// ---------------------------------------------------------------- init / IO
template <typename T>
__global__ void k_init(InstDev I, const double *__restrict__ rho_init, int cur) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= I.N) return;
    T *f = (T *)I.f[cur];
    const long long S = I.S;
    float off[2] = {I.rho0[0], I.rho0[1]};
    if (Store<T>::offset && I.dens[0]) {
        // the state is stored relative to its own densities
        off[0] = (float)rho_init[n];
        off[1] = (float)rho_init[I.N + n];
        I.dens[cur ^ 1][n] = make_float2(off[0], off[1]);
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const double r = rho_init[(long long)s * I.N + n];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double w = i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
            double v = w * r;
            if (Store<T>::offset) v -= w * (double)off[s];
            Store<T>::st(f + (long long)(s * Q + i) * S + n, (float)v);
        }
    }
    float *C = I.C[cur];
    C[n] = 1.f; C[S + n] = 1.f; C[2 * S + n] = 1.f;
    C[3 * S + n] = 0.f; C[4 * S + n] = 0.f; C[5 * S + n] = 0.f;
}

template <typename T>
__global__ void k_decode_pop(InstDev I, int cur, int s, int i, float *dst) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= I.N) return;
    const T *f = (const T *)I.f[cur];
    float v = Store<T>::ld_plain(f + (long long)(s * Q + i) * I.S + n);
    const float2 od = offset_dens<T>(I, cur, n);
    if (Store<T>::offset) v += wq(i) * (s == 0 ? od.x : od.y);
    dst[n] = v;
}

template <typename T>
__global__ void k_encode_pop(InstDev I, int cur, int s, int i, const float *src) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= I.N) return;
    T *f = (T *)I.f[cur];
    float v = src[n];
    const float2 od = offset_dens<T>(I, cur, n);
    if (Store<T>::offset) v -= wq(i) * (s == 0 ? od.x : od.y);
    Store<T>::st(f + (long long)(s * Q + i) * I.S + n, v);
}

// ---------------------------------------------------------------- launchers
cudaError_t launch_moments(const LaunchCtx &c, int cur) {
    switch (c.precision) {
        case LBFE_FP16_OFFSET: k_moments<__half><<<c.total_tiles, kBlock, 0, c.stream>>>(c.inst_dev, c.tile_off, c.n, cur); break;
        case LBFE_BF16_OFFSET: k_moments<__nv_bfloat16><<<c.total_tiles, kBlock, 0, c.stream>>>(c.inst_dev, c.tile_off, c.n, cur); break;
        default: k_moments<float><<<c.total_tiles, kBlock, 0, c.stream>>>(c.inst_dev, c.tile_off, c.n, cur);
    }
    return cudaGetLastError();
}

cudaError_t launch_forces(const LaunchCtx &c, int cur) {
    k_forces<<<c.total_tiles, kBlock, 0, c.stream>>>(c.inst_dev, c.tile_off, c.n, cur);
    return cudaGetLastError();
}

static unsigned nblk(long long N) { return (unsigned)((N + kBlock - 1) / kBlock); }

cudaError_t launch_init(const LaunchCtx &c, int k, const double *rho_dev, int cur) {
    const InstDev &I = c.inst_host[k];
    switch (c.precision) {
        case LBFE_FP16_OFFSET: k_init<__half><<<nblk(I.N), kBlock, 0, c.stream>>>(I, rho_dev, cur); break;
        case LBFE_BF16_OFFSET: k_init<__nv_bfloat16><<<nblk(I.N), kBlock, 0, c.stream>>>(I, rho_dev, cur); break;
        default: k_init<float><<<nblk(I.N), kBlock, 0, c.stream>>>(I, rho_dev, cur);
    }
    return cudaGetLastError();
}

cudaError_t launch_decode_pop(const LaunchCtx &c, int k, int cur, int s, int i, float *dst) {
    const InstDev &I = c.inst_host[k];
    switch (c.precision) {
        case LBFE_FP16_OFFSET: k_decode_pop<__half><<<nblk(I.N), kBlock, 0, c.stream>>>(I, cur, s, i, dst); break;
        case LBFE_BF16_OFFSET: k_decode_pop<__nv_bfloat16><<<nblk(I.N), kBlock, 0, c.stream>>>(I, cur, s, i, dst); break;
        default: k_decode_pop<float><<<nblk(I.N), kBlock, 0, c.stream>>>(I, cur, s, i, dst);
    }
    return cudaGetLastError();
}

cudaError_t launch_encode_pop(const LaunchCtx &c, int k, int cur, int s, int i, const float *src) {
    const InstDev &I = c.inst_host[k];
    switch (c.precision) {
        case LBFE_FP16_OFFSET: k_encode_pop<__half><<<nblk(I.N), kBlock, 0, c.stream>>>(I, cur, s, i, src); break;
        case LBFE_BF16_OFFSET: k_encode_pop<__nv_bfloat16><<<nblk(I.N), kBlock, 0, c.stream>>>(I, cur, s, i, src); break;
        default: k_encode_pop<float><<<nblk(I.N), kBlock, 0, c.stream>>>(I, cur, s, i, src);
    }
    return cudaGetLastError();
}

}  // namespace lbfe
