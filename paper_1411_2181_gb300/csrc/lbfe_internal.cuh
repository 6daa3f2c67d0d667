// lbfe_internal.cuh -- device-side definitions shared by the CUDA
// translation units of liblbfe: the D3Q19 lattice, the storage forms of the
// populations, the per-instance descriptor and the step launchers.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lbfe.h"

namespace lbfe {

constexpr int Q = 19;

// D3Q19 velocity set in the interface order of lbfe.h (rest, 6 faces,
// 12 edges; the opposite of i > 0 is i + 1 for odd i, i - 1 for even i).
__host__ __device__ constexpr int cx(int i) {
    constexpr int t[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return t[i];
}
__host__ __device__ constexpr int cy(int i) {
    constexpr int t[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return t[i];
}
__host__ __device__ constexpr int cz(int i) {
    constexpr int t[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return t[i];
}
// weights 1/3 (rest), 1/18 (faces), 1/36 (edges); c_s^2 = 1/3
__host__ __device__ constexpr float wq(int i) {
    return i == 0 ? 1.0f / 3.0f : (i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

// Storage forms of the populations.  FP32 stores f itself; the reduced
// forms store f - w_i rho0_s rounded to nearest even and decode in FP32.
// ld_l2 reads through L2 only (no L1 allocation): the step kernels keep
// most of the SM's L1/shared capacity as shared memory, and their few
// ordinary loads are throttled when they compete for the small L1.
template <typename T> struct Store;
// st_sr(p, v, r): the store of a time step's populations.  FP32 and FP16
// round to nearest (r unused).  BF16 rounds stochastically: the 16 random
// bits r are added to the FP32 bit pattern below the BF16 mantissa and the
// sum is truncated, so that v rounds up with probability equal to its
// distance from the lower BF16 neighbour in units of the spacing.
// Rounding to nearest repeats the same error in a near-steady state step
// after step; the random bits make the errors average out.
template <> struct Store<float> {
    static constexpr bool offset = false;
    static constexpr bool sround = false;
    static __device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ float ld_l2(const float *p) { return __ldcg(p); }
    static __device__ __forceinline__ float ld_plain(const float *p) { return *p; }
    static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
    static __device__ __forceinline__ void st_sr(float *p, float v, unsigned) { *p = v; }
};
template <> struct Store<__half> {
    static constexpr bool offset = true;
    static constexpr bool sround = false;
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ float ld_l2(const __half *p) { return __half2float(__ldcg(p)); }
    static __device__ __forceinline__ float ld_plain(const __half *p) { return __half2float(*p); }
    static __device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }
    static __device__ __forceinline__ void st_sr(__half *p, float v, unsigned) { *p = __float2half_rn(v); }
};
template <> struct Store<__nv_bfloat16> {
    static constexpr bool offset = true;
    static constexpr bool sround = true;
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ float ld_l2(const __nv_bfloat16 *p) { return __bfloat162float(__ldcg(p)); }
    static __device__ __forceinline__ float ld_plain(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
    static __device__ __forceinline__ void st_sr(__nv_bfloat16 *p, float v, unsigned r16) {
        *reinterpret_cast<unsigned short *>(p) = (unsigned short)((__float_as_uint(v) + (r16 & 0xFFFFu)) >> 16);
    }
};

// Random bits of the stochastic rounding: 32 bits per (destination cell,
// direction, step), the low half for component A and the high half for B;
// the integer hash is "lowbias32" (C. Wellons, hash-prospector), applied to
// the cell and direction mixed with the step by a Weyl constant.
__device__ __forceinline__ unsigned sround_bits(unsigned cell, int dir, unsigned step) {
    unsigned x = (cell * 19u + (unsigned)dir) ^ (step * 0x9E3779B9u);
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// Device descriptor of one instance (all pointers into the caller's block).
struct InstDev {
    int Lx, Ly, Lz, visc_comp;       // visc_comp: 0 (A), 1 (B), -1 Newtonian
    long long N, S;                  // cells, padded stride of one field (multiple of 64)
    void *f[2];                      // populations [2][19][S] in the storage type, ping-pong
    float *C[2];                     // conformation [6][S], ping-pong
    float *rho;                      // scratch [2][S]
    float *jm;                       // scratch [3][S] total momentum
    float *u;                        // scratch [3][S]
    float *F;                        // scratch [2][3][S] per-component total force
    unsigned long long *prof;        // observables: [6][Lx] per-plane integer sums
    double *mpart;                   // observables: [2][kObsBlocks] mass partials
    float G, Uw, nu_A, nu_B;         // Shan-Chen coupling, wall speed, solvent viscosities
    float pi_coef, L2, inv_tauP;     // eta_P/tau_P, L^2, 1/tau_P
    float gx, gy, gz;                // body acceleration
    float rho0[2];                   // constant storage offsets (used when dens is null)
    float2 *dens[2];                 // per-cell offset densities of the reduced forms, ping-pong:
                                     // the state in f[c] is stored relative to w_i * dens[c ^ 1]
    int ntx, nty, nzc, zc;           // fused kernel: column tiles in x, y; z-chunks and their depth
    unsigned *status;                // this instance's status word (may be null)
    unsigned *step_ctr;              // time steps taken, [2] by ping-pong parity (BF16 rounding seed)
};

// Raise a status flag for the whole launch and, when present, for instance I.
__device__ __forceinline__ void raise_flag(unsigned *global, const InstDev &I, unsigned flag) {
    atomicOr(global, flag);
    if (I.status) atomicOr(I.status, flag);
}

constexpr int kBlock = 256;          // threads per block of the cell-per-thread kernels
constexpr int kMaxLx = 4096;         // largest Lx lbfe_derive accepts
constexpr int kObsBlocks = 304;      // 2 x 152 SMs for the observables reduction

__device__ __forceinline__ int wrapi(int a, int L) { return a < 0 ? a + L : (a >= L ? a - L : a); }

// Offset densities (rho0_A, rho0_B) of cell n for the state held in f[cur]:
// the reduced storage forms keep f_i - w_i rho0_s with rho0_s the cell's own
// densities of the previous step (tracked per cell), so that the stored
// value is the small deviation from the cell's rest equilibrium in either
// phase; without tracking the constant offsets apply.  FP32 stores f.
template <typename T>
__device__ __forceinline__ float2 offset_dens(const InstDev &I, int cur, long long n) {
    if (!Store<T>::offset) return make_float2(0.f, 0.f);
    if (I.dens[0]) return __ldg(I.dens[cur ^ 1] + n);
    return make_float2(I.rho0[0], I.rho0[1]);
}

// Instance owning block b of a tiled launch (tile_off[k] = first block of k).
__device__ __forceinline__ int find_inst(const int *tile_off, int n, int b) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(tile_off + mid) <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Peterlin factor f = (L^2 - 3)/(L^2 - tr C) of Eq. 2, evaluated in FP64
// when L^2 - tr C falls below 1e-2 L^2 (close to the extensibility limit).
__device__ __forceinline__ float peterlin(float L2, float cxx, float cyy, float czz) {
    float tr = cxx + cyy + czz;
    float den = L2 - tr;
    if (den < 1e-2f * L2) {
        double dd = (double)L2 - ((double)cxx + (double)cyy + (double)czz);
        return (float)(((double)L2 - 3.0) / dd);
    }
    return (L2 - 3.0f) / den;
}

// Status bits written by the kernels into the handle's status word.
constexpr unsigned kFlagDiverged = 1u;
constexpr unsigned kFlagTimeout = 2u;    // a bounded device-side wait expired (launch status only)

// Launchers (lbfe_fused.cu, lbfe_fields.cu, lbfe_obs.cu).
struct LaunchCtx {
    const InstDev *inst_dev;         // device copy of the descriptors
    const InstDev *inst_host;        // host copy
    const int *tile_off;             // device [n+1]
    int n, total_tiles, precision;
    unsigned *status;                // device status word
    cudaStream_t stream;
    const int *item_off;             // device [n+1]: first fused work item of each instance
    const int *item_off_host;        // host copy of item_off
    int total_items, fused_grid, tile_y;
    int step_kernel;                 // lbfe_step_kernel
    int advection = 0;               // lbfe_params::advection of the batch
    int fused_slots;                 // resident blocks of the fused kernel on the GPU
    const struct PopMaps *maps_host; // per instance: TMA maps of the step kernel (may be null)
    const struct StepMaps *maps_dev; // device copies, [instance][parity]
};
// Tensor maps of the step kernels' TMA copies for one parity of the
// ping-pong state: populations f[b], conformation C[b] and the offset
// densities of the state read (reduced forms).  They live in global memory
// (the handle's block); the launch descriptor points at them.
struct StepMaps {
    CUtensorMap pop;    // box of the tile's own cells (16 rows) or of its radius-2 region (8, 12 rows)
    CUtensorMap c;      // conformation, region box
    CUtensorMap dens;   // offset densities (float2 per cell), region box
};
// Both parities of an instance; ok = 0 when the instance's layout does not
// allow TMA (the kernel then reads with ordinary loads).
struct PopMaps {
    StepMaps m[2];
    int ok;
};
// short_box (test hook): population boxes one row short of what the step
// kernel expects, so that its waits for them expire
cudaError_t fused_pop_maps(const InstDev &I, int precision, int tile_y, bool short_box, PopMaps *m);
cudaError_t launch_fused(const LaunchCtx &c, int cur);
// Kernel launches of one time step of n instances.
int fused_launches(int n);
// Resident blocks per SM of the fused kernel for a tile height.
cudaError_t fused_prepare(int step_kernel, int tile_y, int precision, int advection, int *blocks_per_sm);
cudaError_t launch_moments(const LaunchCtx &c, int cur);
cudaError_t launch_forces(const LaunchCtx &c, int cur);
cudaError_t launch_init(const LaunchCtx &c, int k, const double *rho_dev, int cur);
cudaError_t launch_decode_pop(const LaunchCtx &c, int k, int cur, int s, int i, float *dst);
cudaError_t launch_encode_pop(const LaunchCtx &c, int k, int cur, int s, int i, const float *src);
cudaError_t launch_observables(const LaunchCtx &c, int k, int cur, double *mass_out_dev);

// Host-side droplet analysis (lbfe_analysis.cu): from the observables
// kernel's per-plane sums prof[6][Lx], fill L_p, L_p/2R, necks, fragments,
// broken, volume, centroid, M, D and theta of out.
void droplet_from_profile(const unsigned long long *prof, int Lx, double R, lbfe_obs *out);
void sym_eig3(const double M[6], double ev[3], double V[3][3]);

}  // namespace lbfe
