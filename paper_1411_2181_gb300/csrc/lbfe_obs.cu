// lbfe_obs.cu -- droplet diagnostics (Sec. 1 and Sec. 3: deformation,
// orientation, projected length, necking and break-up).
//
// One pass over the populations of an instance computes, per x-plane, the
// integer sums over the droplet cells (rho_A > rho_B) of 1, y, z, y^2, z^2
// and yz, and the FP64 component masses.  Membership is decided on
// single-precision densities summed in population order.  Each block owns
// the x-columns x = threadIdx.x (mod blockDim.x) of the rows it visits, so
// its shared-memory accumulators need no atomics; blocks merge them into
// global memory with 64-bit integer atomics (exact and order-free).  Masses
// are reduced per block in FP64 and summed in a fixed order by a second
// one-block kernel.  The host turns the per-plane sums into the centroid,
// the second-moment tensor, D, theta, L_p, necks and break-up.
#include "lbfe_internal.cuh"

namespace lbfe {

constexpr int kObsThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kObsThreads)
k_obs_planes(const InstDev *__restrict__ insts, int k, int cur, unsigned *status) {
    const InstDev &I = insts[k];
    extern __shared__ unsigned long long sh[];  // [6][Lx]
    const int Lx = I.Lx, Ly = I.Ly, Lz = I.Lz;
    for (int q = threadIdx.x; q < 6 * Lx; q += blockDim.x) sh[q] = 0ull;
    __syncthreads();
    const T *f = (const T *)I.f[cur];
    const long long S = I.S;
    double mA = 0.0, mB = 0.0;
    bool bad = false;
    const int rows = Ly * Lz;
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const int y = row % Ly, z = row / Ly;
        for (int x = threadIdx.x; x < Lx; x += blockDim.x) {
            const long long n = (long long)row * Lx + x;
            float ra = 0.f, rb = 0.f;
            const float2 od = offset_dens<T>(I, cur, n);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                float va = Store<T>::ld(f + (long long)i * S + n);
                float vb = Store<T>::ld(f + (long long)(Q + i) * S + n);
                if (Store<T>::offset) { va += wq(i) * od.x; vb += wq(i) * od.y; }
                ra += va;
                rb += vb;
            }
            mA += (double)ra;
            mB += (double)rb;
            bad |= (ra != ra) || (rb != rb);
            if (ra > rb) {
                sh[x] += 1ull;
                sh[Lx + x] += (unsigned long long)y;
                sh[2 * Lx + x] += (unsigned long long)z;
                sh[3 * Lx + x] += (unsigned long long)y * y;
                sh[4 * Lx + x] += (unsigned long long)z * z;
                sh[5 * Lx + x] += (unsigned long long)y * z;
            }
        }
    }
    if (bad) raise_flag(status, I, kFlagDiverged);
    __syncthreads();
    for (int q = threadIdx.x; q < 6 * Lx; q += blockDim.x)
        if (sh[q]) atomicAdd(I.prof + q, sh[q]);
    // block reduction of the masses (fixed tree order)
    __shared__ double redA[kObsThreads], redB[kObsThreads];
    redA[threadIdx.x] = mA;
    redB[threadIdx.x] = mB;
    __syncthreads();
    for (int s = kObsThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            redA[threadIdx.x] += redA[threadIdx.x + s];
            redB[threadIdx.x] += redB[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        I.mpart[blockIdx.x] = redA[0];
        I.mpart[kObsBlocks + blockIdx.x] = redB[0];
    }
}

__global__ void k_obs_mass(const InstDev *__restrict__ insts, int k, int nblocks, double *out) {
    const InstDev &I = insts[k];
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < nblocks; ++q) { a += I.mpart[q]; b += I.mpart[kObsBlocks + q]; }
        out[0] = a;
        out[1] = b;
    }
}

cudaError_t launch_observables(const LaunchCtx &c, int k, int cur, double *mass_out_dev) {
    const InstDev &I = c.inst_host[k];
    cudaError_t e = cudaMemsetAsync(I.prof, 0, sizeof(unsigned long long) * 6 * (size_t)I.Lx, c.stream);
    if (e != cudaSuccess) return e;
    const int rows = I.Ly * I.Lz;
    const int nb = rows < kObsBlocks ? rows : kObsBlocks;
    const size_t shmem = sizeof(unsigned long long) * 6 * (size_t)I.Lx;
    switch (c.precision) {
        case LBFE_FP16_OFFSET:
            k_obs_planes<__half><<<nb, kObsThreads, shmem, c.stream>>>(c.inst_dev, k, cur, c.status); break;
        case LBFE_BF16_OFFSET:
            k_obs_planes<__nv_bfloat16><<<nb, kObsThreads, shmem, c.stream>>>(c.inst_dev, k, cur, c.status); break;
        default:
            k_obs_planes<float><<<nb, kObsThreads, shmem, c.stream>>>(c.inst_dev, k, cur, c.status);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_obs_mass<<<1, 32, 0, c.stream>>>(c.inst_dev, k, nb, mass_out_dev);
    return cudaGetLastError();
}

// Dynamic shared memory above 48 KB must be enabled per kernel.
cudaError_t obs_set_smem_limit(size_t bytes) {
    cudaError_t e = cudaFuncSetAttribute(k_obs_planes<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_obs_planes<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_obs_planes<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return e;
}

}  // namespace lbfe
