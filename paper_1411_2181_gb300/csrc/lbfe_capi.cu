// lbfe_capi.cu -- host implementation of the C ABI declared in lbfe.h.
//
// The handle owns no device memory: it carves every field out of the block
// the caller passes to lbfe_create (PyTorch allocates it in the Python
// binding).  All device work is enqueued on the caller's stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lbfe_internal.cuh"

namespace lbfe {
cudaError_t obs_set_smem_limit(size_t bytes);
}

using lbfe::InstDev;

namespace {

thread_local std::string g_cuda_err;

lbfe_status cuda_fail(cudaError_t e, const char *where) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
    g_cuda_err = buf;
    return LBFE_ERR_CUDA;
}

#define CK(call)                                                     \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);          \
    } while (0)

constexpr size_t kAlign = 256;
size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

size_t elem_bytes(int precision) { return precision == LBFE_FP32 ? 4 : 2; }

// NVTX range around a C-ABI call (visible in Nsight Systems / Compute
// timelines; costs a branch when no tool is attached)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

struct Derived {
    double nu_A, nu_B, pi_coef;
    int visc_comp;
};

// Sec. 2: lambda = eta_d/eta_M with total viscosities; DV puts eta_P in the
// droplet (eta_d = eta_A + eta_P, eta_M = eta_B), MV in the matrix
// (eta_d = eta_A, eta_M = eta_B + eta'_P).  Kinematic viscosities use the
// bulk total density rho_in + rho_out.
lbfe_status derive(const lbfe_params &p, Derived &d) {
    if (p.Lx < 1 || p.Ly < 1 || p.Lz < 2 || p.Lx > lbfe::kMaxLx || p.Ly > 65535 || p.Lz > 65535) return LBFE_ERR_BAD_PARAM;
    // the step kernel addresses fields with 32-bit offsets: (s*19 + i)*S + n < 2^32
    if ((long long)p.Lx * p.Ly * p.Lz > (1LL << 26)) return LBFE_ERR_BAD_PARAM;
    if (p.precision < LBFE_FP32 || p.precision > LBFE_BF16_OFFSET) return LBFE_ERR_BAD_PARAM;
    if (p.visco_phase < 0 || p.visco_phase > 2) return LBFE_ERR_BAD_PARAM;
    if (!(p.tau_P > 0.0) || !(p.L2 > 3.0) || !(p.rho_in > 0.0) || !(p.rho_out >= 0.0)) return LBFE_ERR_BAD_PARAM;
    if (!(std::fabs(p.Uw) < 0.1) || !(p.eta_M > 0.0) || !(p.lambda > 0.0) || !(p.eta_P >= 0.0)) return LBFE_ERR_BAD_PARAM;
    if (!(p.G >= 0.0)) return LBFE_ERR_BAD_PARAM;
    if (p.advection != LBFE_ADVECTION_UPWIND1 && p.advection != LBFE_ADVECTION_UPWIND2_MINMOD) return LBFE_ERR_BAD_PARAM;
    const double rho_ref = p.rho_in + p.rho_out;
    const double eta_d = p.lambda * p.eta_M;
    double eta_A = eta_d, eta_B = p.eta_M;
    d.pi_coef = 0.0;
    d.visc_comp = -1;
    if (p.visco_phase == LBFE_DROPLET_VISCOELASTIC) {
        eta_A = eta_d - p.eta_P;
        d.pi_coef = p.eta_P / p.tau_P;
        d.visc_comp = 0;
    } else if (p.visco_phase == LBFE_MATRIX_VISCOELASTIC) {
        eta_B = p.eta_M - p.eta_P;
        d.pi_coef = p.eta_P / p.tau_P;
        d.visc_comp = 1;
    }
    d.nu_A = eta_A / rho_ref;
    d.nu_B = eta_B / rho_ref;
    if (!(d.nu_A > 0.0) || !(d.nu_B > 0.0)) return LBFE_ERR_BAD_PARAM;
    return LBFE_OK;
}

struct Layout {
    size_t inst_off, tile_off, item_off, status_off, mass_off, maps_off;
    std::vector<size_t> f_off[2], C_off[2], scratch_off, prof_off, mpart_off, dens_off;
    size_t total;
};

long long stride_of(const lbfe_params &p) {
    const long long N = (long long)p.Lx * p.Ly * p.Lz;
    return (N + 63) / 64 * 64;
}

Layout plan(const lbfe_params *p, int n) {
    Layout L;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, kAlign); return o; };
    L.inst_off = take(sizeof(InstDev) * (size_t)n);
    L.tile_off = take(sizeof(int) * (size_t)(n + 1));
    L.item_off = take(sizeof(int) * (size_t)(n + 1));
    // launch word, work counters, then one status word per instance and
    // two step-count words per instance (by ping-pong parity)
    L.status_off = take(sizeof(unsigned) * (4 + 3 * (size_t)n));
    L.mass_off = take(sizeof(double) * 2);
    L.maps_off = take(sizeof(lbfe::StepMaps) * 2 * (size_t)n);   // TMA maps, [instance][parity]
    const size_t eb = elem_bytes(p[0].precision);
    for (int k = 0; k < n; ++k) {
        const size_t S = (size_t)stride_of(p[k]);
        L.f_off[0].push_back(take(eb * 2 * lbfe::Q * S));
        L.f_off[1].push_back(take(eb * 2 * lbfe::Q * S));
        L.C_off[0].push_back(take(sizeof(float) * 6 * S));
        L.C_off[1].push_back(take(sizeof(float) * 6 * S));
        L.scratch_off.push_back(take(sizeof(float) * 14 * S));
        L.prof_off.push_back(take(sizeof(unsigned long long) * 6 * (size_t)p[k].Lx));
        L.mpart_off.push_back(take(sizeof(double) * 2 * lbfe::kObsBlocks));
        // reduced storage forms: per-cell offset densities, ping-pong
        L.dens_off.push_back(p[0].precision == LBFE_FP32 ? 0 : take(sizeof(float) * 2 * 2 * S));
    }
    L.total = off;
    return L;
}

}  // namespace

struct lbfe_handle {
    int n = 0, precision = 0;
    cudaStream_t stream = nullptr;
    std::vector<lbfe_params> params;
    std::vector<InstDev> inst;
    std::vector<long long> steps;
    std::vector<char> ready;
    char *base = nullptr;
    Layout layout;
    InstDev *inst_dev = nullptr;
    int *tile_off = nullptr;
    int total_tiles = 0;
    int *item_off = nullptr;
    std::vector<int> item_off_h;
    std::vector<lbfe::PopMaps> maps;
    lbfe::StepMaps *maps_dev = nullptr;
    int total_items = 0, fused_grid = 0, tile_y = 16, z_chunk_req = 0, num_sms = 0, blocks_per_sm = 0;
    int step_kernel = LBFE_STEP_CELL;
    int advection = 0;               // lbfe_params::advection of every instance
    unsigned inject = 0;             // lbfe_test_inject bits
    unsigned *status = nullptr;
    double *mass = nullptr;
    int cur = 0;
    // CUDA graphs of one time step from each parity of the ping-pong state,
    // captured on a private stream and replayed by lbfe_step; dropped when
    // the launch shape changes
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t step_graph[2] = {nullptr, nullptr};

    void drop_graphs() {
        for (auto &g : step_graph)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
    }

    lbfe::LaunchCtx ctx() const {
        lbfe::LaunchCtx c;
        c.inst_dev = inst_dev;
        c.inst_host = inst.data();
        c.tile_off = tile_off;
        c.n = n;
        c.total_tiles = total_tiles;
        c.precision = precision;
        c.status = status;
        c.stream = stream;
        c.item_off = item_off;
        c.item_off_host = item_off_h.data();
        c.maps_host = maps.empty() ? nullptr : maps.data();
        c.maps_dev = maps_dev;
        c.fused_slots = num_sms * blocks_per_sm;
        c.total_items = total_items;
        c.fused_grid = fused_grid;
        c.tile_y = tile_y;
        c.step_kernel = step_kernel;
        c.advection = advection;
        return c;
    }
};

// Work items of the fused kernel: per instance ceil(Lx/32) x ceil(Ly/TY)
// column tiles times nzc z-chunks.  Without a requested chunk depth, nzc is
// chosen so that the items fill the resident blocks of the GPU about once
// (chunks of at least 8 planes).
static lbfe_status configure_fused(lbfe_handle *h, int step_kernel, int tile_y, int z_chunk) {
    if (step_kernel == LBFE_STEP_PAIR) {
        if (tile_y != 16) return LBFE_ERR_BAD_PARAM;
        for (auto &I : h->inst)
            if (I.Lx % 2) return LBFE_ERR_BAD_PARAM;
    } else if (step_kernel != LBFE_STEP_CELL || (tile_y != 8 && tile_y != 12 && tile_y != 16)) {
        return LBFE_ERR_BAD_PARAM;
    }
    if (z_chunk < 0) return LBFE_ERR_BAD_PARAM;
    // the second-order advection scheme has the one-cell kernel at 8 rows only
    if (h->advection != 0 && (step_kernel != LBFE_STEP_CELL || tile_y != 8)) return LBFE_ERR_BAD_PARAM;
    int bps = 0;
    cudaError_t e = lbfe::fused_prepare(step_kernel, tile_y, h->precision, h->advection, &bps);
    if (e != cudaSuccess) return cuda_fail(e, "fused_prepare");
    if (bps < 1) return LBFE_ERR_BAD_PARAM;
    long long columns = 0;
    for (auto &I : h->inst) {
        I.ntx = (I.Lx + 31) / 32;
        I.nty = (I.Ly + tile_y - 1) / tile_y;
        columns += (long long)I.ntx * I.nty;
    }
    const long long slots = (long long)h->num_sms * bps;
    std::vector<int> off(h->n + 1, 0);
    for (int k = 0; k < h->n; ++k) {
        InstDev &I = h->inst[k];
        int zc = z_chunk;
        if (zc == 0) {
            long long nz = (slots + columns / 2) / columns;
            if (nz < 1) nz = 1;
            zc = (int)((I.Lz + nz - 1) / nz);
            if (zc < 8) zc = 8;
        }
        if (zc > I.Lz) zc = I.Lz;
        I.zc = zc;
        I.nzc = (I.Lz + zc - 1) / zc;
        const long long items = (long long)I.ntx * I.nty * I.nzc;
        if (off[k] + items > (long long)0x7fffffff) return LBFE_ERR_BAD_PARAM;
        off[k + 1] = off[k] + (int)items;
    }
    h->drop_graphs();
    h->tile_y = tile_y;
    h->step_kernel = step_kernel;
    h->z_chunk_req = z_chunk;
    h->blocks_per_sm = bps;
    h->total_items = off[h->n];
    h->item_off_h = off;
    h->maps.assign(h->n, lbfe::PopMaps{});
    std::vector<lbfe::StepMaps> md(2 * (size_t)h->n);
    for (int k = 0; k < h->n; ++k) {
        e = lbfe::fused_pop_maps(h->inst[k], h->precision, tile_y, (h->inject & LBFE_INJECT_SHORT_COPIES) != 0,
                                 &h->maps[k]);
        if (e != cudaSuccess) return cuda_fail(e, "fused_pop_maps");
        md[2 * k] = h->maps[k].m[0];
        md[2 * k + 1] = h->maps[k].m[1];
    }
    e = cudaMemcpyAsync(h->maps_dev, md.data(), sizeof(lbfe::StepMaps) * md.size(), cudaMemcpyHostToDevice,
                        h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "configure_fused");
    h->fused_grid = (int)std::min<long long>(h->total_items, slots);
    e = cudaMemcpyAsync(h->inst_dev, h->inst.data(), sizeof(InstDev) * h->n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->item_off, off.data(), sizeof(int) * (h->n + 1), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "configure_fused");
    return LBFE_OK;
}

extern "C" {

const char *lbfe_status_str(lbfe_status s) {
    switch (s) {
        case LBFE_OK: return "ok";
        case LBFE_ERR_BAD_PARAM: return "invalid argument or parameters";
        case LBFE_ERR_NO_MEMORY: return "device block smaller than required";
        case LBFE_ERR_CUDA: return "CUDA runtime error";
        case LBFE_ERR_DIVERGED: return "simulation diverged";
        case LBFE_ERR_TIMEOUT: return "device wait timed out";
        case LBFE_ERR_STATE: return "call out of order";
        case LBFE_ERR_IO: return "checkpoint file unreadable, unwritable or corrupt";
    }
    return "unknown status";
}

const char *lbfe_last_cuda_error(void) { return g_cuda_err.c_str(); }
size_t lbfe_params_size(void) { return sizeof(lbfe_params); }
size_t lbfe_obs_size(void) { return sizeof(lbfe_obs); }

lbfe_status lbfe_derive(const lbfe_params *p, lbfe_derived *out) {
    if (!p) return LBFE_ERR_BAD_PARAM;
    Derived d;
    lbfe_status s = derive(*p, d);
    if (s != LBFE_OK) return s;
    const double tauA = 3.0 * d.nu_A + 0.5, tauB = 3.0 * d.nu_B + 0.5;
    if (!(tauA > 0.5) || !(tauB > 0.5)) return LBFE_ERR_BAD_PARAM;
    if (out) {
        out->nu_A = d.nu_A;
        out->nu_B = d.nu_B;
        out->tau_A = tauA;
        out->tau_B = tauB;
        out->pi_coef = d.pi_coef;
        out->gamma_dot = 2.0 * p->Uw / p->Lz;
        out->Ca = p->sigma > 0 ? p->eta_M * out->gamma_dot * p->R / p->sigma : 0.0;
        out->tau_em = p->sigma > 0 ? p->R * p->eta_M / p->sigma : 0.0;
        out->De = out->tau_em > 0 ? (p->tau_P / out->tau_em) * (p->eta_P / p->eta_M) : 0.0;
        // Eq. 7: N1 = 8 (eta_P/tau_P)(L^2/6) sinh^2(asinh(gdot tau_P L^2/4 (L^2/6)^(-3/2)) / 3)
        const double gd = std::fabs(out->gamma_dot), l6 = p->L2 / 6.0;
        const double sh = std::sinh(std::asinh(gd * p->tau_P * p->L2 / 4.0 * std::pow(l6, -1.5)) / 3.0);
        const double N1 = 8.0 * (p->eta_P / p->tau_P) * l6 * sh * sh;
        const double Ca = std::fabs(out->Ca);
        out->De_N1 = Ca > 0 ? N1 * p->R / (2.0 * p->sigma * Ca * Ca) : 0.0;
    }
    return LBFE_OK;
}

lbfe_status lbfe_required_bytes(const lbfe_params *p, int n, size_t *bytes) {
    if (!p || n < 1 || !bytes) return LBFE_ERR_BAD_PARAM;
    for (int k = 0; k < n; ++k) {
        lbfe_status s = lbfe_derive(p + k, nullptr);
        if (s != LBFE_OK) return s;
        if (p[k].precision != p[0].precision || p[k].advection != p[0].advection) return LBFE_ERR_BAD_PARAM;
    }
    *bytes = plan(p, n).total;
    return LBFE_OK;
}

lbfe_status lbfe_create(lbfe_handle **hp, const lbfe_params *p, int n, void *device_block, size_t bytes,
                        void *stream) {
    if (!hp) return LBFE_ERR_BAD_PARAM;
    *hp = nullptr;
    size_t need = 0;
    lbfe_status s = lbfe_required_bytes(p, n, &need);
    if (s != LBFE_OK) return s;
    if (!device_block || ((uintptr_t)device_block % kAlign) != 0) return LBFE_ERR_BAD_PARAM;
    if (bytes < need) return LBFE_ERR_NO_MEMORY;
    lbfe_handle *h = new (std::nothrow) lbfe_handle;
    if (!h) return LBFE_ERR_NO_MEMORY;
    h->n = n;
    h->precision = p[0].precision;
    h->advection = p[0].advection;
    h->stream = (cudaStream_t)stream;
    h->params.assign(p, p + n);
    h->steps.assign(n, 0);
    h->ready.assign(n, 0);
    h->base = (char *)device_block;
    h->layout = plan(p, n);
    const Layout &L = h->layout;
    h->inst_dev = (InstDev *)(h->base + L.inst_off);
    h->tile_off = (int *)(h->base + L.tile_off);
    h->item_off = (int *)(h->base + L.item_off);
    h->status = (unsigned *)(h->base + L.status_off);
    h->mass = (double *)(h->base + L.mass_off);
    h->maps_dev = (lbfe::StepMaps *)(h->base + L.maps_off);
    std::vector<int> toff(n + 1, 0);
    int maxLx = 0;
    for (int k = 0; k < n; ++k) {
        Derived d;
        derive(p[k], d);
        InstDev I;
        memset(&I, 0, sizeof I);
        I.Lx = p[k].Lx; I.Ly = p[k].Ly; I.Lz = p[k].Lz;
        I.visc_comp = d.visc_comp;
        I.N = (long long)p[k].Lx * p[k].Ly * p[k].Lz;
        I.S = stride_of(p[k]);
        I.f[0] = h->base + L.f_off[0][k];
        I.f[1] = h->base + L.f_off[1][k];
        I.C[0] = (float *)(h->base + L.C_off[0][k]);
        I.C[1] = (float *)(h->base + L.C_off[1][k]);
        float *scr = (float *)(h->base + L.scratch_off[k]);
        I.rho = scr;
        I.jm = scr + 2 * I.S;
        I.u = scr + 5 * I.S;
        I.F = scr + 8 * I.S;
        I.prof = (unsigned long long *)(h->base + L.prof_off[k]);
        I.status = h->status + 4 + k;
        I.step_ctr = h->status + 4 + n + 2 * k;
        I.mpart = (double *)(h->base + L.mpart_off[k]);
        I.G = (float)p[k].G;
        I.Uw = (float)p[k].Uw;
        I.nu_A = (float)d.nu_A;
        I.nu_B = (float)d.nu_B;
        I.pi_coef = (float)d.pi_coef;
        I.L2 = (float)p[k].L2;
        I.inv_tauP = (float)(1.0 / p[k].tau_P);
        I.gx = (float)p[k].g[0]; I.gy = (float)p[k].g[1]; I.gz = (float)p[k].g[2];
        I.rho0[0] = (float)p[k].rho0[0];
        I.rho0[1] = (float)p[k].rho0[1];
        if (p[0].precision != LBFE_FP32) {
            I.dens[0] = (float2 *)(h->base + L.dens_off[k]);
            I.dens[1] = I.dens[0] + I.S;
        }
        h->inst.push_back(I);
        toff[k + 1] = toff[k] + (int)((I.N + lbfe::kBlock - 1) / lbfe::kBlock);
        if (p[k].Lx > maxLx) maxLx = p[k].Lx;
    }
    h->total_tiles = toff[n];
    cudaError_t e = cudaMemcpyAsync(h->inst_dev, h->inst.data(), sizeof(InstDev) * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->tile_off, toff.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->status, 0, sizeof(unsigned) * (4 + 3 * (size_t)n), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    const size_t smem = sizeof(unsigned long long) * 6 * (size_t)maxLx;
    if (e == cudaSuccess && smem > 48 * 1024) e = lbfe::obs_set_smem_limit(smem);
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "lbfe_create");
    }
    // default shape: the one the autotuner picks for the 192 x 96 x 80
    // workload on most GB300s (8-row tiles in FP32, 12-row with 2-byte storage)
    lbfe_status st =
        configure_fused(h, LBFE_STEP_CELL, (h->precision == LBFE_FP32 || h->advection != 0) ? 8 : 12, 0);
    if (st != LBFE_OK) {
        delete h;
        return st;
    }
    *hp = h;
    return LBFE_OK;
}

lbfe_status lbfe_init(lbfe_handle *h, int k, const double *rho_init) {
    const NvtxRange nvtx_range("lbfe_init");
    if (!h || k < 0 || k >= h->n || !rho_init) return LBFE_ERR_BAD_PARAM;
    const InstDev &I = h->inst[k];
    // stage the densities (FP64) in the instance's scratch, then build f^eq
    double *stage = (double *)I.rho;
    CK(cudaMemcpyAsync(stage, rho_init, sizeof(double) * 2 * (size_t)I.N, cudaMemcpyHostToDevice, h->stream));
    CK(lbfe::launch_init(h->ctx(), k, stage, h->cur));
    CK(cudaMemsetAsync(I.status, 0, sizeof(unsigned), h->stream));
    CK(cudaMemsetAsync(I.step_ctr, 0, 2 * sizeof(unsigned), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->steps[k] = 0;
    h->ready[k] = 1;
    return LBFE_OK;
}

// Capture the launches of one step from state parity cur into a graph.
static cudaError_t build_step_graph(lbfe_handle *h, int cur) {
    cudaError_t e = cudaSuccess;
    if (!h->cap_stream) e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    lbfe::LaunchCtx c = h->ctx();
    c.stream = h->cap_stream;
    const cudaError_t el = lbfe::launch_fused(c, cur);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(h->cap_stream, &g);
    if (el != cudaSuccess) e = el;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->step_graph[cur], g, 0);
    if (g) cudaGraphDestroy(g);
    return e;
}

lbfe_status lbfe_step(lbfe_handle *h, long long nsteps) {
    const NvtxRange nvtx_range("lbfe_step");
    if (!h || nsteps < 0) return LBFE_ERR_BAD_PARAM;
    for (int k = 0; k < h->n; ++k)
        if (!h->ready[k]) return LBFE_ERR_STATE;
    // runs of several steps replay captured graphs (no per-launch argument
    // marshalling); inside a caller's own stream capture, or for a single
    // step, the kernels are launched directly
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(h->stream, &cs));
    const bool graphs = nsteps >= 2 && cs == cudaStreamCaptureStatusNone;
    const lbfe::LaunchCtx c = h->ctx();
    for (long long t = 0; t < nsteps; ++t) {
        if (graphs) {
            if (!h->step_graph[h->cur]) CK(build_step_graph(h, h->cur));
            CK(cudaGraphLaunch(h->step_graph[h->cur], h->stream));
        } else {
            CK(lbfe::launch_fused(c, h->cur));
        }
        h->cur ^= 1;
    }
    for (int k = 0; k < h->n; ++k) h->steps[k] += nsteps;
    return LBFE_OK;
}

lbfe_status lbfe_check(lbfe_handle *h) {
    if (!h) return LBFE_ERR_BAD_PARAM;
    unsigned st = 0;
    CK(cudaMemcpyAsync(&st, h->status, sizeof st, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (st & lbfe::kFlagTimeout) return LBFE_ERR_TIMEOUT;
    return (st & lbfe::kFlagDiverged) ? LBFE_ERR_DIVERGED : LBFE_OK;
}

lbfe_status lbfe_observables(lbfe_handle *h, int k, lbfe_obs *out) {
    const NvtxRange nvtx_range("lbfe_observables");
    if (!h || k < 0 || k >= h->n || !out) return LBFE_ERR_BAD_PARAM;
    if (!h->ready[k]) return LBFE_ERR_STATE;
    const InstDev &I = h->inst[k];
    const lbfe_params &p = h->params[k];
    CK(lbfe::launch_observables(h->ctx(), k, h->cur, h->mass));
    std::vector<unsigned long long> prof(6 * (size_t)I.Lx);
    double mass[2];
    unsigned st = 0;
    CK(cudaMemcpyAsync(prof.data(), I.prof, sizeof(unsigned long long) * prof.size(), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(mass, h->mass, sizeof mass, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(&st, I.status, sizeof st, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));

    memset(out, 0, sizeof *out);
    out->step = h->steps[k];
    out->mass[0] = mass[0];
    out->mass[1] = mass[1];
    out->flags = (int)st;
    const double tem = p.sigma > 0 ? p.R * p.eta_M / p.sigma : 0.0;
    out->t_over_tem = tem > 0 ? (double)h->steps[k] / tem : 0.0;
    lbfe::droplet_from_profile(prof.data(), I.Lx, p.R, out);
    return (st & lbfe::kFlagDiverged) ? LBFE_ERR_DIVERGED : LBFE_OK;
}

lbfe_status lbfe_get_field(lbfe_handle *h, int k, int which, void *host_dst, size_t bytes) {
    if (!h || k < 0 || k >= h->n || !host_dst) return LBFE_ERR_BAD_PARAM;
    if (!h->ready[k]) return LBFE_ERR_STATE;
    const InstDev &I = h->inst[k];
    const size_t N = (size_t)I.N, S = (size_t)I.S;
    float *dst = (float *)host_dst;
    const lbfe::LaunchCtx c = h->ctx();
    switch (which) {
        case LBFE_FIELD_F: {
            if (bytes != sizeof(float) * 2 * lbfe::Q * N) return LBFE_ERR_BAD_PARAM;
            float *tmp = I.u;  // scratch slice of >= N floats
            for (int s = 0; s < 2; ++s)
                for (int i = 0; i < lbfe::Q; ++i) {
                    CK(lbfe::launch_decode_pop(c, k, h->cur, s, i, tmp));
                    CK(cudaMemcpyAsync(dst + (size_t)(s * lbfe::Q + i) * N, tmp, sizeof(float) * N,
                                       cudaMemcpyDeviceToHost, h->stream));
                    CK(cudaStreamSynchronize(h->stream));
                }
            return LBFE_OK;
        }
        case LBFE_FIELD_C:
            if (bytes != sizeof(float) * 6 * N) return LBFE_ERR_BAD_PARAM;
            CK(cudaMemcpy2DAsync(dst, sizeof(float) * N, I.C[h->cur], sizeof(float) * S, sizeof(float) * N, 6,
                                 cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            return LBFE_OK;
        case LBFE_FIELD_RHO:
        case LBFE_FIELD_U: {
            const int rows = which == LBFE_FIELD_RHO ? 2 : 3;
            if (bytes != sizeof(float) * rows * N) return LBFE_ERR_BAD_PARAM;
            CK(lbfe::launch_moments(c, h->cur));
            if (which == LBFE_FIELD_U) CK(lbfe::launch_forces(c, h->cur));
            const float *src = which == LBFE_FIELD_RHO ? I.rho : I.u;
            CK(cudaMemcpy2DAsync(dst, sizeof(float) * N, src, sizeof(float) * S, sizeof(float) * N, rows,
                                 cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            return LBFE_OK;
        }
        default:
            return LBFE_ERR_BAD_PARAM;
    }
}

lbfe_status lbfe_set_field(lbfe_handle *h, int k, int which, const void *host_src, size_t bytes) {
    if (!h || k < 0 || k >= h->n || !host_src) return LBFE_ERR_BAD_PARAM;
    if (!h->ready[k]) return LBFE_ERR_STATE;
    const InstDev &I = h->inst[k];
    const size_t N = (size_t)I.N, S = (size_t)I.S;
    const float *src = (const float *)host_src;
    switch (which) {
        case LBFE_FIELD_F: {
            if (bytes != sizeof(float) * 2 * lbfe::Q * N) return LBFE_ERR_BAD_PARAM;
            float *tmp = I.u;
            const lbfe::LaunchCtx c = h->ctx();
            if (I.dens[0]) {
                // the new state is stored relative to its own densities
                std::vector<float2> d(N);
                for (size_t n = 0; n < N; ++n) {
                    float a = 0.f, b = 0.f;
                    for (int i = 0; i < lbfe::Q; ++i) {
                        a += src[(size_t)i * N + n];
                        b += src[(size_t)(lbfe::Q + i) * N + n];
                    }
                    d[n] = make_float2(a, b);
                }
                CK(cudaMemcpyAsync(I.dens[h->cur ^ 1], d.data(), sizeof(float2) * N, cudaMemcpyHostToDevice,
                                   h->stream));
                CK(cudaStreamSynchronize(h->stream));
            }
            for (int s = 0; s < 2; ++s)
                for (int i = 0; i < lbfe::Q; ++i) {
                    CK(cudaMemcpyAsync(tmp, src + (size_t)(s * lbfe::Q + i) * N, sizeof(float) * N,
                                       cudaMemcpyHostToDevice, h->stream));
                    CK(lbfe::launch_encode_pop(c, k, h->cur, s, i, tmp));
                    CK(cudaStreamSynchronize(h->stream));
                }
            return LBFE_OK;
        }
        case LBFE_FIELD_C:
            if (bytes != sizeof(float) * 6 * N) return LBFE_ERR_BAD_PARAM;
            CK(cudaMemcpy2DAsync(I.C[h->cur], sizeof(float) * S, src, sizeof(float) * N, sizeof(float) * N, 6,
                                 cudaMemcpyHostToDevice, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            return LBFE_OK;
        default:
            return LBFE_ERR_BAD_PARAM;
    }
}

int lbfe_launches_per_step(const lbfe_handle *h) { return h ? lbfe::fused_launches(h->n) : 0; }

// Column blocks (x-split domain decomposition): the stored state of
// x-columns [x0, x0 + nx) as [38][Lz][Ly][nx] populations in the storage
// type, [6][Lz][Ly][nx] FP32 conformation and, in the reduced forms,
// [Lz][Ly][nx] offset-density pairs; copied as stored, so that a block moved
// between instances keeps every bit.
static size_t column_bytes(const lbfe_handle *h, const InstDev &I, int nx) {
    const size_t cells = (size_t)nx * I.Ly * I.Lz;
    return cells * (2 * lbfe::Q * elem_bytes(h->precision) + 6 * sizeof(float) +
                    (h->precision == LBFE_FP32 ? 0 : sizeof(float2)));
}

lbfe_status lbfe_columns_bytes(const lbfe_handle *h, int k, int nx, size_t *bytes) {
    if (!h || k < 0 || k >= h->n || !bytes || nx < 1 || nx > h->inst[k].Lx) return LBFE_ERR_BAD_PARAM;
    *bytes = column_bytes(h, h->inst[k], nx);
    return LBFE_OK;
}

static lbfe_status copy_columns(lbfe_handle *h, int k, int x0, int nx, char *dev, bool get) {
    if (!h || k < 0 || k >= h->n || !dev || nx < 1 || x0 < 0) return LBFE_ERR_BAD_PARAM;
    const InstDev &I = h->inst[k];
    if (x0 + nx > I.Lx) return LBFE_ERR_BAD_PARAM;
    if (!h->ready[k]) return LBFE_ERR_STATE;
    const size_t rows = (size_t)I.Ly * I.Lz, S = (size_t)I.S;
    const size_t eb = elem_bytes(h->precision);
    auto copy = [&](char *field, size_t esz, size_t count, size_t fstride, size_t &off) -> cudaError_t {
        for (size_t a = 0; a < count; ++a) {
            char *f = field + (a * fstride + (size_t)x0) * esz;
            char *b = dev + off;
            const cudaError_t e =
                get ? cudaMemcpy2DAsync(b, nx * esz, f, I.Lx * esz, nx * esz, rows, cudaMemcpyDeviceToDevice, h->stream)
                    : cudaMemcpy2DAsync(f, I.Lx * esz, b, nx * esz, nx * esz, rows, cudaMemcpyDeviceToDevice, h->stream);
            if (e != cudaSuccess) return e;
            off += rows * nx * esz;
        }
        return cudaSuccess;
    };
    size_t off = 0;
    // the current state: populations f[cur], conformation C[cur] and the
    // offsets the populations are stored against (dens[cur ^ 1])
    CK(copy((char *)I.f[h->cur], eb, 2 * lbfe::Q, S, off));
    CK(copy((char *)I.C[h->cur], sizeof(float), 6, S, off));
    if (h->precision != LBFE_FP32 && I.dens[0]) CK(copy((char *)I.dens[h->cur ^ 1], sizeof(float2), 1, 0, off));
    return LBFE_OK;
}

lbfe_status lbfe_get_columns(lbfe_handle *h, int k, int x0, int nx, void *dev_dst) {
    return copy_columns(h, k, x0, nx, (char *)dev_dst, true);
}

lbfe_status lbfe_set_columns(lbfe_handle *h, int k, int x0, int nx, const void *dev_src) {
    return copy_columns(h, k, x0, nx, (char *)const_cast<void *>(dev_src), false);
}

lbfe_status lbfe_test_inject(lbfe_handle *h, unsigned what) {
    if (!h || (what & ~(unsigned)LBFE_INJECT_SHORT_COPIES)) return LBFE_ERR_BAD_PARAM;
    CK(cudaStreamSynchronize(h->stream));
    h->inject = what;
    // rebuild the tensor maps of the current launch shape
    return configure_fused(h, h->step_kernel, h->tile_y, h->z_chunk_req);
}

lbfe_status lbfe_tune(lbfe_handle *h, int step_kernel, int tile_y, int z_chunk) {
    if (!h) return LBFE_ERR_BAD_PARAM;
    return configure_fused(h, step_kernel, tile_y, z_chunk);
}

lbfe_status lbfe_launch_config(const lbfe_handle *h, int *step_kernel, int *tile_y, int *z_chunk, int *grid,
                               int *items) {
    if (!h) return LBFE_ERR_BAD_PARAM;
    if (step_kernel) *step_kernel = h->step_kernel;
    if (tile_y) *tile_y = h->tile_y;
    if (z_chunk) *z_chunk = h->inst[0].zc;
    if (grid) *grid = h->fused_grid;
    if (items) *items = h->total_items;
    return LBFE_OK;
}

unsigned lbfe_crc32(const void *data, size_t n, unsigned crc) {
    // table-driven CRC-32, reflected polynomial 0xEDB88320
    static unsigned table[256];
    static std::once_flag once;
    std::call_once(once, [] {
        for (unsigned i = 0; i < 256; ++i) {
            unsigned c = i;
            for (int b = 0; b < 8; ++b) c = (c & 1u) ? 0xEDB88320u ^ (c >> 1) : c >> 1;
            table[i] = c;
        }
    });
    const unsigned char *p = static_cast<const unsigned char *>(data);
    crc = ~crc;
    for (size_t i = 0; i < n; ++i) crc = table[(crc ^ p[i]) & 0xFFu] ^ (crc >> 8);
    return ~crc;
}

namespace {

// Checkpoint file: this header, then populations, C and offset densities.
struct CkptHeader {
    char magic[8];                   // "LBFECKPT"
    unsigned version;                // 1
    unsigned header_bytes;           // sizeof(CkptHeader)
    lbfe_params params;
    long long steps, cells;
    unsigned precision, elem_bytes;
    unsigned long long f_bytes, c_bytes, d_bytes;
    unsigned payload_crc;
    unsigned header_crc;             // CRC of the header with this field zero
};
constexpr char kCkptMagic[8] = {'L', 'B', 'F', 'E', 'C', 'K', 'P', 'T'};

unsigned header_crc(CkptHeader hd) {
    hd.header_crc = 0;
    return lbfe_crc32(&hd, sizeof hd, 0);
}

struct FileCloser {
    FILE *f;
    ~FileCloser() {
        if (f) std::fclose(f);
    }
};

}  // namespace

lbfe_status lbfe_save(lbfe_handle *h, int k, const char *path) {
    const NvtxRange nvtx_range("lbfe_save");
    if (!h || !path || k < 0 || k >= h->n) return LBFE_ERR_BAD_PARAM;
    if (!h->ready[k]) return LBFE_ERR_STATE;
    const InstDev &I = h->inst[k];
    const size_t N = (size_t)I.N, S = (size_t)I.S, eb = elem_bytes(h->precision);
    const bool dens = h->precision != LBFE_FP32 && I.dens[0] != nullptr;
    CkptHeader hd{};
    std::memcpy(hd.magic, kCkptMagic, 8);
    hd.version = 1;
    hd.header_bytes = sizeof hd;
    hd.params = h->params[k];
    hd.steps = h->steps[k];
    hd.cells = I.N;
    hd.precision = (unsigned)h->precision;
    hd.elem_bytes = (unsigned)eb;
    hd.f_bytes = 2ull * lbfe::Q * N * eb;
    hd.c_bytes = 6ull * N * sizeof(float);
    hd.d_bytes = dens ? N * sizeof(float2) : 0ull;
    std::vector<char> buf(hd.f_bytes + hd.c_bytes + hd.d_bytes);
    char *fb = buf.data(), *cb = fb + hd.f_bytes, *db = cb + hd.c_bytes;
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaMemcpy2DAsync(fb, N * eb, I.f[h->cur], S * eb, N * eb, 2 * lbfe::Q, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpy2DAsync(cb, N * sizeof(float), I.C[h->cur], S * sizeof(float), N * sizeof(float), 6,
                         cudaMemcpyDeviceToHost, h->stream));
    // the state in f[cur] is stored relative to the offset densities dens[cur ^ 1]
    if (dens) CK(cudaMemcpyAsync(db, I.dens[h->cur ^ 1], hd.d_bytes, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    hd.payload_crc = lbfe_crc32(buf.data(), buf.size(), 0);
    hd.header_crc = header_crc(hd);
    FileCloser fc{std::fopen(path, "wb")};
    if (!fc.f) return LBFE_ERR_IO;
    if (std::fwrite(&hd, sizeof hd, 1, fc.f) != 1) return LBFE_ERR_IO;
    if (!buf.empty() && std::fwrite(buf.data(), buf.size(), 1, fc.f) != 1) return LBFE_ERR_IO;
    const int rc = std::fclose(fc.f);
    fc.f = nullptr;
    return rc == 0 ? LBFE_OK : LBFE_ERR_IO;
}

lbfe_status lbfe_load(lbfe_handle *h, int k, const char *path) {
    const NvtxRange nvtx_range("lbfe_load");
    if (!h || !path || k < 0 || k >= h->n) return LBFE_ERR_BAD_PARAM;
    InstDev &I = h->inst[k];
    const size_t N = (size_t)I.N, S = (size_t)I.S, eb = elem_bytes(h->precision);
    const bool dens = h->precision != LBFE_FP32 && I.dens[0] != nullptr;
    FileCloser fc{std::fopen(path, "rb")};
    if (!fc.f) return LBFE_ERR_IO;
    CkptHeader hd{};
    if (std::fread(&hd, sizeof hd, 1, fc.f) != 1) return LBFE_ERR_IO;
    if (std::memcmp(hd.magic, kCkptMagic, 8) != 0 || hd.version != 1 || hd.header_bytes != sizeof hd ||
        hd.header_crc != header_crc(hd))
        return LBFE_ERR_IO;
    if (std::memcmp(&hd.params, &h->params[k], sizeof hd.params) != 0 || hd.cells != I.N ||
        hd.precision != (unsigned)h->precision || hd.elem_bytes != eb)
        return LBFE_ERR_BAD_PARAM;
    if (hd.f_bytes != 2ull * lbfe::Q * N * eb || hd.c_bytes != 6ull * N * sizeof(float) ||
        hd.d_bytes != (dens ? N * sizeof(float2) : 0ull))
        return LBFE_ERR_IO;
    std::vector<char> buf(hd.f_bytes + hd.c_bytes + hd.d_bytes);
    if (!buf.empty() && std::fread(buf.data(), buf.size(), 1, fc.f) != 1) return LBFE_ERR_IO;
    if (lbfe_crc32(buf.data(), buf.size(), 0) != hd.payload_crc) return LBFE_ERR_IO;
    const char *fb = buf.data(), *cb = fb + hd.f_bytes, *db = cb + hd.c_bytes;
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaMemcpy2DAsync(I.f[h->cur], S * eb, fb, N * eb, N * eb, 2 * lbfe::Q, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpy2DAsync(I.C[h->cur], S * sizeof(float), cb, N * sizeof(float), N * sizeof(float), 6,
                         cudaMemcpyHostToDevice, h->stream));
    if (dens) CK(cudaMemcpyAsync(I.dens[h->cur ^ 1], db, hd.d_bytes, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemsetAsync(I.status, 0, sizeof(unsigned), h->stream));
    // the step count seeds the BF16 stochastic rounding: a resumed run
    // continues with the random bits of an uninterrupted one
    const unsigned step_ctr = (unsigned)hd.steps;
    CK(cudaMemcpyAsync(I.step_ctr + h->cur, &step_ctr, sizeof step_ctr, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->steps[k] = hd.steps;
    h->ready[k] = 1;
    return LBFE_OK;
}

lbfe_status lbfe_destroy(lbfe_handle *h) {
    if (!h) return LBFE_ERR_BAD_PARAM;
    cudaStreamSynchronize(h->stream);
    h->drop_graphs();
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    delete h;
    return LBFE_OK;
}

}  // extern "C"
