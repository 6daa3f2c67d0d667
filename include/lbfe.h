/*
 * lbfe.h -- C ABI of the GB300 hybrid lattice-Boltzmann / FENE-P droplet
 * solver (Gupta & Sbragaglia, "Deformation and break-up of viscoelastic
 * droplets using Lattice Boltzmann Models").
 *
 * The problem (Sec. 3, set-up; Fig. 1 sketch): a droplet of component A
 * with radius R between two walls at gap W = Lz moving at -Uw (bottom,
 * z = -1/2) and +Uw (top, z = Lz - 1/2) along x, periodic in x and y, in a
 * matrix of component B.  Immiscibility is Shan-Chen (Sec. 2); the
 * total-viscosity ratio is lambda (Sec. 2); one phase may carry FENE-P
 * polymers (Eqs. 1-4) with viscosity eta_P, relaxation time tau_P and
 * extensibility L^2 (Sec. 2).  The observables are deformation, orientation,
 * projected length, neck count and break-up (Secs. 1 and 3, Figs. 2-4).
 *
 * Memory: the caller owns every buffer.  Device memory is one block the
 * caller allocates (any CUDA allocator, e.g. PyTorch's) of at least the size
 * lbfe_required_bytes() reports, 256-byte aligned, and keeps alive until
 * lbfe_destroy(); the library carves its fields out of it and allocates no
 * device memory of its own.  Host pointers are read or written only during
 * the call that receives them.  All device work is enqueued on the CUDA
 * stream given at creation (NULL = legacy default stream); calls that
 * return host data synchronise that stream.
 *
 * Errors: every call returns an lbfe_status and never aborts, traps or
 * exits.  A numerical blow-up (non-positive or NaN density, tr C >= L^2) is
 * flagged on the device by the step kernels, per instance, and reported as
 * LBFE_ERR_DIVERGED by the next lbfe_observables() of that instance (and by
 * lbfe_check() for any instance of the handle).
 *
 * Field layout (the interface format of lbfe_get_field / lbfe_set_field):
 *   cell index n = (z*Ly + y)*Lx + x, N = Lx*Ly*Lz;
 *   populations f[(s*19 + i)*N + n], s = 0 (A, droplet), 1 (B, matrix);
 *   D3Q19 order i: 0 rest; 1..6 = +x,-x,+y,-y,+z,-z;
 *   7..18 = (1,1,0),(-1,-1,0),(1,-1,0),(-1,1,0),(1,0,1),(-1,0,-1),
 *           (1,0,-1),(-1,0,1),(0,1,1),(0,-1,-1),(0,1,-1),(0,-1,1);
 *   conformation C[k*N + n], k = xx, yy, zz, xy, xz, yz.
 * The populations are the post-streaming (pre-collision) state.
 */
#ifndef LBFE_H
#define LBFE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBFE_OK = 0,
    LBFE_ERR_BAD_PARAM = 1,   /* invalid argument or parameter set (nothing enqueued) */
    LBFE_ERR_NO_MEMORY = 2,   /* the device block given is smaller than required */
    LBFE_ERR_CUDA = 3,        /* a CUDA runtime call failed (see lbfe_last_cuda_error) */
    LBFE_ERR_DIVERGED = 4,    /* the device flagged a numerical blow-up */
    LBFE_ERR_TIMEOUT = 5,     /* a bounded device-side wait expired */
    LBFE_ERR_STATE = 6,       /* call out of order, e.g. step before init */
    LBFE_ERR_IO = 7           /* checkpoint file unreadable, unwritable, truncated or corrupt */
} lbfe_status;

typedef enum {
    LBFE_FP32 = 0,            /* populations stored in FP32 */
    LBFE_FP16_OFFSET = 1,     /* stored as FP16 offsets f - w_i rho_s', FP32 compute */
    LBFE_BF16_OFFSET = 2      /* stored as BF16 offsets f - w_i rho_s', FP32 compute; rho_s' is
                                 the cell's own density of the previous step, kept in FP32.
                                 The step's stores round stochastically, with random bits
                                 drawn from the destination cell, the direction and the
                                 instance's step count (deterministic: a run, a batch member
                                 and a run resumed by lbfe_load give the same bits); FP16
                                 rounds to nearest */
} lbfe_precision;

typedef enum {
    LBFE_NEWTONIAN = 0,
    LBFE_DROPLET_VISCOELASTIC = 1,  /* DV: polymer in component A */
    LBFE_MATRIX_VISCOELASTIC = 2    /* MV: polymer in component B */
} lbfe_visco_phase;

/* Parameters of one droplet instance (lattice units). */
/* Discretisation of u . grad C in the FENE-P update (the paper defers its
 * FD scheme).  UPWIND1: first-order upwind.  UPWIND2_MINMOD: second-order
 * upwind with minmod-limited slopes (face values reconstructed from the
 * upwind side); runs with the one-cell step kernel at 8-row tiles only. */
typedef enum {
    LBFE_ADVECTION_UPWIND1 = 0,
    LBFE_ADVECTION_UPWIND2_MINMOD = 1
} lbfe_advection;

typedef struct {
    int Lx, Ly, Lz;           /* lattice; the wall gap W is Lz */
    int visco_phase;          /* lbfe_visco_phase */
    int precision;            /* lbfe_precision (the same for every instance of a batch) */
    int advection;            /* lbfe_advection of u.grad C (the same for every instance of a batch) */
    double R;                 /* droplet radius at rest: reference length of L_p/2R and Ca */
    double Uw;                /* wall speed; shear rate 2 Uw / W */
    double G;                 /* Shan-Chen inter-component coupling (> 0 separates) */
    double eta_M;             /* matrix total dynamic viscosity */
    double lambda;            /* droplet/matrix total-viscosity ratio (Sec. 2) */
    double eta_P;             /* polymer viscosity of the viscoelastic phase */
    double tau_P;             /* polymer relaxation time (> 0) */
    double L2;                /* FENE-P extensibility L^2 (> 3) */
    double rho_in;            /* bulk density of a component where it is the majority */
    double rho_out;           /* bulk density of the dissolved component */
    double sigma;             /* interfacial tension of G (bookkeeping of Ca, De, tau_em) */
    double g[3];              /* constant body acceleration (verification hook; 0 normally) */
    double rho0[2];           /* constant offsets of the reduced forms in lbfe_observables_noalloc */
} lbfe_params;

/* Derived numbers (host arithmetic only). */
typedef struct {
    double nu_A, nu_B;        /* solvent kinematic viscosities */
    double tau_A, tau_B;      /* BGK relaxation times in the two bulk phases */
    double pi_coef;           /* eta_P / tau_P of the viscoelastic phase */
    double gamma_dot;         /* 2 Uw / W (Sec. 3) */
    double Ca;                /* eta_M gamma_dot R / sigma (Sec. 1) */
    double tau_em;            /* R eta_M / sigma, Eq. 9 */
    double De;                /* (tau_P / tau_em)(eta_P / eta_M), Eq. 8 */
    double De_N1;             /* N1 R / (2 sigma Ca^2), Eq. 5, with the steady-shear
                                 N1 of Eq. 7 at this shear rate; equals De in the
                                 Oldroyd-B limit L^2 -> infinity */
} lbfe_derived;

/* Droplet observables of one instance. */
typedef struct {
    long long step;           /* steps taken since lbfe_init */
    double mass[2];           /* sum of rho_A and rho_B over the box (FP64) */
    double volume;            /* number of droplet cells (rho_A > rho_B) */
    double centroid[3];       /* droplet centroid; x in [0, Lx) */
    double M[6];              /* second moments about the centroid: xx, yy, zz, xy, xz, yz */
    double D;                 /* (a - b)/(a + b), a, b from the extreme eigenvalues of M */
    double theta_deg;         /* major-axis angle from +x in the x-z plane, (-90, 90] */
    double Lp;                /* projected length on x (occupied planes, periodic) */
    double Lp_over_2R;        /* Lp / (2 R) */
    double t_over_tem;        /* step / tau_em */
    int necks;                /* interior non-empty minima of the x-profile below half the adjacent maxima */
    int fragments;            /* separated occupied x-runs holding >= 1% of the volume */
    int broken;               /* fragments >= 2 */
    int flags;                /* this instance's device status word (bit 0: diverged) */
} lbfe_obs;

typedef struct lbfe_handle lbfe_handle;

/* Fields for lbfe_get_field / lbfe_set_field (float32 host arrays). */
enum {
    LBFE_FIELD_F = 0,         /* populations [2][19][N] (decoded to FP32); get and set */
    LBFE_FIELD_C = 1,         /* conformation [6][N]; get and set */
    LBFE_FIELD_RHO = 2,       /* densities [2][N] of the current state; get only */
    LBFE_FIELD_U = 3          /* velocity (j + F/2)/rho [3][N] of the current state; get only */
};

const char *lbfe_status_str(lbfe_status s);
/* Message of the last failing CUDA call in this thread ("" if none). */
const char *lbfe_last_cuda_error(void);
/* sizeof() of the structs, so that bindings can check their marshalling. */
size_t lbfe_params_size(void);
size_t lbfe_obs_size(void);

/* Validate p and fill the derived numbers.  BAD_PARAM on: a non-positive
 * lattice size, Lz < 2, Lx > 4096, Ly or Lz > 65535, more than 2^26 cells in one instance
 * (larger boxes: split into a batch), a solvent viscosity <= 0 (eta_P too large), BGK
 * tau <= 1/2, tau_P <= 0, L^2 <= 3, Uw >= 0.1 (Mach limit), an unknown
 * phase or precision.  out may be NULL. */
lbfe_status lbfe_derive(const lbfe_params *p, lbfe_derived *out);

/* Device bytes needed by a batch of n instances with parameters p[0..n-1]. */
lbfe_status lbfe_required_bytes(const lbfe_params *p, int n, size_t *bytes);

/* Create a solver over n instances (n = 1 for a single droplet).  p is
 * copied; device_block (>= lbfe_required_bytes, 256-byte aligned) is
 * borrowed until lbfe_destroy; stream is a cudaStream_t or NULL.  All
 * instances of a batch share p[0].precision. */
lbfe_status lbfe_create(lbfe_handle **h, const lbfe_params *p, int n, void *device_block,
                        size_t bytes, void *stream);

/* Initial state of instance k from host densities rho_init[2][N] (float64):
 * f = f^eq(rho_s, u = 0) and C = I (Sec. 3: droplet at rest when the walls
 * start).  Resets the step counter.  Copies synchronously from host memory. */
lbfe_status lbfe_init(lbfe_handle *h, int k, const double *rho_init);

/* Advance every instance by nsteps time steps of the hybrid scheme (Sec. 2:
 * the two-component lattice-Boltzmann collide + stream with the Shan-Chen
 * force, the per-site relaxation time of the viscosity ratio and the
 * moving walls of Sec. 3, coupled to the finite-difference FENE-P update of
 * C (Eqs. 2 and 4) and to the polymer-stress divergence of Eqs. 1 and 3),
 * asynchronously on the stream.
 * With nsteps >= 2 the steps replay CUDA graphs of one step (captured once
 * per launch shape on a private stream); results are identical to single
 * steps.  Inside a stream capture of the caller the kernels are launched
 * directly into it. */
lbfe_status lbfe_step(lbfe_handle *h, long long nsteps);

/* Observables of instance k (synchronises the stream). */
lbfe_status lbfe_observables(lbfe_handle *h, int k, lbfe_obs *out);

/* TIMEOUT if a bounded device-side wait of the step kernel expired (a TMA
 * copy that did not complete in time; the kernel finishes without it and
 * the step's result is invalid), else DIVERGED if any instance has flagged a
 * blow-up, else OK (synchronises). */
lbfe_status lbfe_check(lbfe_handle *h);

/* Copy a field of instance k to / from host memory (float32; bytes must be
 * exactly the field's size).  Synchronises the stream. */
lbfe_status lbfe_get_field(lbfe_handle *h, int k, int which, void *host_dst, size_t bytes);
lbfe_status lbfe_set_field(lbfe_handle *h, int k, int which, const void *host_src, size_t bytes);

/* Column blocks of an instance, for a domain split along x (not in the
 * paper, whose lattices fit one machine; it gives the way to larger
 * lattices over several GPUs).  A block is the stored current state of the
 * x-columns [x0, x0 + nx): populations [38][Lz][Ly][nx] in the storage type
 * (FP32, or the FP16 / BF16 offsets), conformation [6][Lz][Ly][nx] FP32 and,
 * in the reduced forms, the per-cell offset densities [Lz][Ly][nx] as FP32
 * pairs, contiguous in that order, copied bit for bit.  A slab that
 * carries two ghost columns on each side, filled before every step with the
 * neighbouring slabs' edge columns, advances its interior columns exactly
 * as the undivided lattice does: every stencil of the step (Shan-Chen
 * force, polymer-stress divergence, velocity gradient, streaming) reaches
 * at most two cells, and the ghosts' own results are discarded.
 *   lbfe_columns_bytes  size of a block of nx columns of instance k;
 *   lbfe_get_columns    copy columns [x0, x0 + nx) into the device buffer
 *                       dev_dst (device to device, asynchronous on the
 *                       handle's stream);
 *   lbfe_set_columns    copy a block from dev_src into columns [x0, x0 + nx).
 * BAD_PARAM for columns outside [0, Lx) or a null pointer, STATE before
 * lbfe_init.  The buffers are the caller's (at least lbfe_columns_bytes). */
lbfe_status lbfe_columns_bytes(const lbfe_handle *h, int k, int nx, size_t *bytes);
lbfe_status lbfe_get_columns(lbfe_handle *h, int k, int x0, int nx, void *dev_dst);
lbfe_status lbfe_set_columns(lbfe_handle *h, int k, int x0, int nx, const void *dev_src);

/* Number of kernel launches one lbfe_step(h, 1) enqueues: one per group of
 * up to 64 instances (the step kernel carries the instance descriptors in
 * its parameter space). */
int lbfe_launches_per_step(const lbfe_handle *h);

/* Variants of the time-step kernel.  Both compute the same step (results
 * agree to FP32 rounding); they differ in speed only. */
typedef enum {
    LBFE_STEP_CELL = 0,   /* one cell per thread, tiles of 32 x tile_y cells, tile_y in {8, 12, 16} */
    LBFE_STEP_PAIR = 1    /* two x-adjacent cells per thread, 32 x 16 tiles; needs even Lx everywhere */
} lbfe_step_kernel;

/* Launch shape of the step kernel: variant (lbfe_step_kernel), column-tile
 * height tile_y (tile width 32; 16 for LBFE_STEP_PAIR) and z-chunk depth in
 * planes (0 = automatic: fill the resident blocks of the GPU about once).
 * A new handle starts with LBFE_STEP_CELL, tile_y 8 (FP32, or any precision
 * with LBFE_ADVECTION_UPWIND2_MINMOD) or 12 (FP16 / BF16 storage) and the
 * automatic z-chunk.  With LBFE_ADVECTION_UPWIND2_MINMOD only
 * LBFE_STEP_CELL at tile_y 8 is accepted.
 * LBFE_ERR_BAD_PARAM for an unsupported combination.  Synchronises the
 * stream. */
lbfe_status lbfe_tune(lbfe_handle *h, int step_kernel, int tile_y, int z_chunk);
/* Current launch shape (any output may be NULL): kernel variant, tile
 * height, z-chunk of instance 0, persistent grid size and number of work
 * items. */
lbfe_status lbfe_launch_config(const lbfe_handle *h, int *step_kernel, int *tile_y, int *z_chunk, int *grid,
                               int *items);

/* Test hook for the failure path of the step kernel (no counterpart in the
 * paper).  what = LBFE_INJECT_SHORT_COPIES: the TMA tensor maps of the
 * populations are rebuilt with boxes one row short of what the step kernel
 * expects, so that the completion barrier of each block's first copy never
 * completes.  Each thread's bounded wait expires (after about one second of
 * GPU time); from then on it waits for no copy and the block's issuing
 * thread issues none, the block runs through its work items on stale data
 * (the step's result is invalid), waits once more (bounded) for the barrier
 * of the last copy it issued, frees its tensor memory and exits;
 * lbfe_check then reports LBFE_ERR_TIMEOUT (the launch status word keeps the
 * flag for the life of the handle).  Only instances whose staging uses TMA
 * (Lx * element size a multiple of 16 bytes) wait.  what = 0 restores the
 * maps.  Synchronises the stream; BAD_PARAM for unknown bits. */
#define LBFE_INJECT_SHORT_COPIES 1u
lbfe_status lbfe_test_inject(lbfe_handle *h, unsigned what);

/* Observables of a population field the caller already holds on the
 * device, computed without allocating anything.  For callers that cannot
 * allocate device memory at the point where they want diagnostics: their
 * memory belongs to another allocator whose pool must not be bypassed, they
 * run under a device-memory budget fixed at start-up, or they cannot afford
 * the device-wide synchronisation of cudaFree in a latency-sensitive loop.
 * The paper has no counterpart of this entry point.
 *   p       parameters of the field (sizes, precision, storage offsets rho0;
 *           validated as in lbfe_derive);
 *   f_dev   device pointer to populations [2][19][stride] in the storage
 *           type of p->precision, in the layout and order of this header.
 *           FP32: the populations themselves.  FP16 / BF16: f_i - w_i rho0_s
 *           with the CONSTANT offsets p->rho0[s]; the solver's own reduced
 *           state is stored against per-cell offset densities instead and
 *           cannot be decoded here (use lbfe_observables for it, or pass
 *           its FP32 populations from lbfe_get_field);
 *   stride  elements between population arrays, >= Lx*Ly*Lz;
 *   out     host result (same fields and readings as lbfe_observables;
 *           step and t_over_tem are 0);
 *   stream  cudaStream_t or NULL; synchronised before return.
 * Scratch lives in a file-scope device array of about 200 KB that every
 * GPU loading the library keeps until the process exits.  It holds the
 * per-plane sums of up to 4096 x-planes, which covers every Lx that
 * lbfe_derive accepts (larger Lx returns LBFE_ERR_BAD_PARAM from that
 * validation, before any device work).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it; make that first call before any
 * stream capture.  Every call shares the array and it keeps the last
 * call's contents (each call clears what must start at zero).  Host calls
 * are serialised and each synchronises its stream, so calls made through
 * this function do not overlap; calls that did overlap on the GPU would race
 * on the shared array.  Calls no cudaMalloc, cudaFree or other allocating
 * routine. */
lbfe_status lbfe_observables_noalloc(const lbfe_params *p, const void *f_dev, long long stride, lbfe_obs *out,
                                     void *stream);

/* Checkpoint / resume of instance k (not in the paper: its runs are single
 * long integrations).  lbfe_save writes the instance's state after its last
 * step: the parameter set, the step count, the populations (the storage
 * type, [2][19][N] without the stride padding), C ([6][N] float32) and, in
 * the reduced forms, the per-cell offset densities ([N] pairs of float32),
 * into one raw little-endian file at path, behind a header that carries a
 * CRC-32 of itself and one of the payload (lbfe_crc32).  lbfe_load reads such
 * a file into instance k of a handle created with the same parameter set
 * (compared byte for byte: BAD_PARAM otherwise) and makes it ready to step;
 * resumed runs are bitwise identical to uninterrupted ones at the same
 * launch shape.  IO for a file that cannot be opened, read or written, is
 * truncated, or fails a CRC.  Both synchronise the stream; BAD_PARAM for a
 * null handle or path or k out of range, STATE for lbfe_save before
 * lbfe_init. */
lbfe_status lbfe_save(lbfe_handle *h, int k, const char *path);
lbfe_status lbfe_load(lbfe_handle *h, int k, const char *path);

/* CRC-32 (reflected polynomial 0xEDB88320, the one of zlib and PNG) of n
 * bytes, continuing from crc (0 to start); host only. */
unsigned lbfe_crc32(const void *data, size_t n, unsigned crc);

/* Release the handle (the device block stays the caller's). */
lbfe_status lbfe_destroy(lbfe_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* LBFE_H */
