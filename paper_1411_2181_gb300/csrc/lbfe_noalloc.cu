// lbfe_noalloc.cu -- droplet observables of a caller-owned population field
// without any allocation.
//
// Some callers cannot allocate device memory when they want diagnostics:
// their memory is entirely owned by another allocator whose pool must not
// be bypassed, they run under a fixed device-memory budget reserved at
// start-up, or they cannot afford the device-wide synchronisation that
// cudaFree implies in a latency-sensitive loop.  For them this entry point
// computes the observables of a population field they already hold, with
// its scratch (the per-plane sums, the mass partials, the status word and a
// copy of the field descriptor) in a file-scope device array that every GPU
// loading this library keeps until the process exits.  It calls no
// cudaMalloc, cudaFree or other allocating routine.
#include <cstring>
#include <mutex>

#include "lbfe_internal.cuh"

namespace lbfe {
cudaError_t obs_set_smem_limit(size_t bytes);
}

namespace {

constexpr int kScratchMaxLx = 4096;       // largest Lx the static scratch holds
// lbfe_derive rejects Lx > lbfe::kMaxLx first; the scratch covers every
// Lx it accepts
static_assert(kScratchMaxLx >= lbfe::kMaxLx, "static scratch smaller than the accepted Lx range");
constexpr int kMaxDevices = 64;

// Layout of the static scratch (8-byte words):
//   [0, 6*kScratchMaxLx)           per-plane integer sums
//   next 2*kObsBlocks              FP64 mass partials
//   next 2                          FP64 masses
//   next 1                          status word (low 32 bits)
//   next ceil(sizeof(InstDev)/8)    field descriptor
constexpr size_t kProfWords = 6 * (size_t)kScratchMaxLx;
constexpr size_t kPartWords = 2 * (size_t)lbfe::kObsBlocks;
constexpr size_t kDescWords = (sizeof(lbfe::InstDev) + 7) / 8;
constexpr size_t kScratchWords = kProfWords + kPartWords + 2 + 1 + kDescWords;

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kScratchWords];

std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the static scratch on the current device, looked up
// once per device (the host-side symbol is not a device address).
lbfe_status scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBFE_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return LBFE_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return LBFE_OK;
}

// Host copy of the per-plane sums (no allocation per call; guarded by the
// same mutex for the whole call).
unsigned long long g_host_prof[kProfWords];
std::mutex g_call_mutex;

}  // namespace

extern "C" lbfe_status lbfe_observables_noalloc(const lbfe_params *p, const void *f_dev, long long stride,
                                                 lbfe_obs *out, void *stream) {
    if (!p || !f_dev || !out) return LBFE_ERR_BAD_PARAM;
    lbfe_derived d;
    lbfe_status st = lbfe_derive(p, &d);
    if (st != LBFE_OK) return st;
    if (p->Lx > kScratchMaxLx) return LBFE_ERR_BAD_PARAM;    // beyond the static scratch
    const long long N = (long long)p->Lx * p->Ly * p->Lz;
    if (stride < N) return LBFE_ERR_BAD_PARAM;
    void *base = nullptr;
    st = scratch_address(&base);
    if (st != LBFE_OK) return st;
    std::lock_guard<std::mutex> lock(g_call_mutex);
    cudaStream_t s = (cudaStream_t)stream;

    unsigned long long *words = (unsigned long long *)base;
    lbfe::InstDev I;
    memset(&I, 0, sizeof I);
    I.Lx = p->Lx;
    I.Ly = p->Ly;
    I.Lz = p->Lz;
    I.N = N;
    I.S = stride;
    I.f[0] = const_cast<void *>(f_dev);
    I.prof = words;
    I.mpart = (double *)(words + kProfWords);
    I.rho0[0] = (float)p->rho0[0];
    I.rho0[1] = (float)p->rho0[1];
    double *mass_dev = (double *)(words + kProfWords + kPartWords);
    unsigned *status_dev = (unsigned *)(words + kProfWords + kPartWords + 2);
    lbfe::InstDev *desc_dev = (lbfe::InstDev *)(words + kProfWords + kPartWords + 3);

    lbfe::LaunchCtx c;
    memset(&c, 0, sizeof c);
    c.inst_dev = desc_dev;
    c.inst_host = &I;
    c.n = 1;
    c.precision = p->precision;
    c.status = status_dev;
    c.stream = s;
    cudaError_t e = cudaMemsetAsync(status_dev, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(desc_dev, &I, sizeof I, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        const size_t smem = sizeof(unsigned long long) * 6 * (size_t)p->Lx;
        if (smem > 48 * 1024) e = lbfe::obs_set_smem_limit(smem);
    }
    if (e == cudaSuccess) e = lbfe::launch_observables(c, 0, 0, mass_dev);  // clears the plane sums itself
    double mass[2] = {0.0, 0.0};
    unsigned status = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g_host_prof, words, sizeof(unsigned long long) * 6 * (size_t)p->Lx,
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(mass, mass_dev, sizeof mass, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, status_dev, sizeof status, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return LBFE_ERR_CUDA;

    memset(out, 0, sizeof *out);
    out->mass[0] = mass[0];
    out->mass[1] = mass[1];
    out->flags = (int)status;
    lbfe::droplet_from_profile(g_host_prof, p->Lx, p->R, out);
    return (status & lbfe::kFlagDiverged) ? LBFE_ERR_DIVERGED : LBFE_OK;
}
