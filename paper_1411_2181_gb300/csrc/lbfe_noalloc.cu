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
#include <cmath>
#include <cstring>
#include <mutex>

#include "lbfe_internal.cuh"

namespace lbfe {
cudaError_t obs_set_smem_limit(size_t bytes);
}

namespace {

constexpr int kMaxLx = 4096;              // largest Lx the static scratch holds
constexpr int kMaxDevices = 64;

// Layout of the static scratch (8-byte words):
//   [0, 6*kMaxLx)                  per-plane integer sums
//   next 2*kObsBlocks              FP64 mass partials
//   next 2                          FP64 masses
//   next 1                          status word (low 32 bits)
//   next ceil(sizeof(InstDev)/8)    field descriptor
constexpr size_t kProfWords = 6 * (size_t)kMaxLx;
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

// Host-side analysis of the per-plane sums (same readings as the handle
// API: longest empty circular run -> L_p and the unwrapped x origin;
// interior non-empty minima below half the adjacent maxima -> necks;
// occupied runs with >= 1% of the volume -> fragments).
struct ProfileResult {
    int Lp, start, necks, frags;
};

ProfileResult profile_of(const unsigned long long *A, int Lx) {
    ProfileResult r{0, 0, 0, 0};
    unsigned long long V = 0;
    for (int x = 0; x < Lx; ++x) V += A[x];
    if (V == 0) return r;
    int best = 0, best_end = 0;
    for (int x = 0; x < Lx; ++x) {
        if (A[x] != 0 || A[(x + Lx - 1) % Lx] == 0) continue;
        int len = 0;
        while (len < Lx && A[(x + len) % Lx] == 0) ++len;
        if (len > best) { best = len; best_end = x + len; }
    }
    r.start = best > 0 ? best_end % Lx : 0;
    r.Lp = Lx - best;
    unsigned long long run = 0;
    long long prev_max = -1, dip = 0, last = 0;
    bool have_dip = false, rising = true;
    for (int q = 0; q <= r.Lp; ++q) {
        const long long a = q < r.Lp ? (long long)A[(r.start + q) % Lx] : 0;
        if (a != 0) {
            run += (unsigned long long)a;
        } else if (run) {
            if (100 * run >= V) ++r.frags;
            run = 0;
        }
        if (a == last) continue;                 // plateau: keep its first plane
        if (a < last && rising) {                // `last` was a local maximum
            if (have_dip && prev_max >= 0 && dip > 0 && 2 * dip < (prev_max < last ? prev_max : last)) ++r.necks;
            prev_max = last;
            have_dip = false;
        } else if (a > last && !rising) {        // `last` was a local minimum
            dip = last;
            have_dip = true;
        }
        rising = a > last;
        last = a;
    }
    return r;
}

// Eigen-decomposition of a symmetric 3x3 matrix by cyclic Jacobi sweeps.
void eig_sym3(const double m[6], double ev[3], double vec[3][3]) {
    double a[3][3] = {{m[0], m[3], m[4]}, {m[3], m[1], m[5]}, {m[4], m[5], m[2]}};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) vec[i][j] = i == j;
    for (int sweep = 0; sweep < 50; ++sweep) {
        if (std::fabs(a[0][1]) + std::fabs(a[0][2]) + std::fabs(a[1][2]) == 0.0) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (a[p][q] == 0.0) continue;
                const double th = 0.5 * std::atan2(2.0 * a[p][q], a[q][q] - a[p][p]);
                const double c = std::cos(th), s = std::sin(th);
                for (int k = 0; k < 3; ++k) {
                    const double kp = a[k][p], kq = a[k][q];
                    a[k][p] = c * kp - s * kq;
                    a[k][q] = s * kp + c * kq;
                }
                for (int k = 0; k < 3; ++k) {
                    const double pk = a[p][k], qk = a[q][k];
                    a[p][k] = c * pk - s * qk;
                    a[q][k] = s * pk + c * qk;
                }
                for (int k = 0; k < 3; ++k) {
                    const double kp = vec[k][p], kq = vec[k][q];
                    vec[k][p] = c * kp - s * kq;
                    vec[k][q] = s * kp + c * kq;
                }
            }
    }
    for (int i = 0; i < 3; ++i) ev[i] = a[i][i];
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
    if (p->Lx > kMaxLx) return LBFE_ERR_BAD_PARAM;    // beyond the static scratch
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
    const int Lx = p->Lx;
    const unsigned long long *A = g_host_prof;
    const ProfileResult pr = profile_of(A, Lx);
    out->Lp = pr.Lp;
    out->Lp_over_2R = p->R > 0 ? pr.Lp / (2.0 * p->R) : 0.0;
    out->necks = pr.necks;
    out->fragments = pr.frags;
    out->broken = pr.frags >= 2;
    double V = 0, sx = 0, sxx = 0, sy = 0, sz = 0, syy = 0, szz = 0, syz = 0, sxy = 0, sxz = 0;
    for (int x = 0; x < Lx; ++x) {
        const double xp = (double)((x - pr.start + Lx) % Lx), a = (double)A[x];
        V += a;
        sx += xp * a;
        sxx += xp * xp * a;
        sy += (double)A[Lx + x];
        sz += (double)A[2 * Lx + x];
        syy += (double)A[3 * Lx + x];
        szz += (double)A[4 * Lx + x];
        syz += (double)A[5 * Lx + x];
        sxy += xp * (double)A[Lx + x];
        sxz += xp * (double)A[2 * Lx + x];
    }
    out->volume = V;
    if (V > 0) {
        const double cx = sx / V, cy = sy / V, cz = sz / V;
        out->centroid[0] = std::fmod(cx + pr.start, (double)Lx);
        out->centroid[1] = cy;
        out->centroid[2] = cz;
        double *M = out->M;
        M[0] = sxx - V * cx * cx; M[1] = syy - V * cy * cy; M[2] = szz - V * cz * cz;
        M[3] = sxy - V * cx * cy; M[4] = sxz - V * cx * cz; M[5] = syz - V * cy * cz;
        double ev[3], vec[3][3];
        eig_sym3(M, ev, vec);
        int imax = 0, imin = 0;
        for (int q = 1; q < 3; ++q) {
            if (ev[q] > ev[imax]) imax = q;
            if (ev[q] < ev[imin]) imin = q;
        }
        const double a = std::sqrt(5.0 * std::fmax(ev[imax], 0.0) / V);
        const double b = std::sqrt(5.0 * std::fmax(ev[imin], 0.0) / V);
        out->D = (a + b) > 0 ? (a - b) / (a + b) : 0.0;
        double th = std::atan2(vec[2][imax], vec[0][imax]) * 180.0 / M_PI;
        if (th <= -90.0) th += 180.0;
        if (th > 90.0) th -= 180.0;
        out->theta_deg = th;
    }
    return (status & lbfe::kFlagDiverged) ? LBFE_ERR_DIVERGED : LBFE_OK;
}
