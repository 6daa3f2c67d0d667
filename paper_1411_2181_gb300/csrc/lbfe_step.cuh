// lbfe_step.cuh -- device building blocks of the time-step kernels
// (lbfe_fused.cu: one cell per thread; lbfe_fused2.cu: two x-adjacent cells
// per thread): launch descriptors, TMEM / TMA / mbarrier access, the
// shared-memory rings and the per-cell stage functions.
//
// One time step of the hybrid LBM / FENE-P method (Sec. 2) runs as a single
// persistent kernel that reads every population and conformation component
// once and writes it once.
//
// Work decomposition.  A work item is a column tile of 32 x TY cells in the
// x-y plane over a chunk [z0, z1) of planes of one instance.  Block b starts
// with item b; launches with more items than blocks hand out the rest from
// a counter.  Inside an item the block marches along z with shared-memory
// rings holding, per plane, the fields the stencils need:
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
// Two block barriers per plane: after stage M, and after stage U.  Stages
// X(p-1) and U(p-2) need, from stage F(p-1), only the thread's own cell
// (forces and u of the collision; u of plane p-1 in the z-derivative of
// grad u), so they follow stage F without a barrier; the x- and
// y-derivatives of stage U use u of plane p-2, complete since the previous
// plane.
// Planes beyond a wall are loaded as the adjacent plane (mirror ghosts of
// rho, C and Pi); the velocity ghost 2 U_wall - u is applied in stage U.
//
// Blackwell specifics.
//  * TMA staging: one elected thread copies the next plane into a shared
//    staging buffer as soon as stage M has consumed it, so the DRAM reads of
//    plane p+1 overlap stages F, X and U of plane p; completion is tracked by
//    an mbarrier with a bounded wait.  Tiles of up to 12 rows copy their
//    whole radius-2 region (populations, conformation and, in the reduced
//    storage forms, the offset densities: one box each); tiles
//    of 16 rows copy their own cells and read the halo with ordinary loads.
//    Cells across a periodic seam and ragged-tile cells use ordinary loads
//    (through L2 only: the large shared carve-out leaves little L1).  For
//    FP32 8-row tiles the next copy starts once every thread has read the
//    staging buffer (a second mbarrier), before the stage-M barrier.
//  * TMEM handoff: each thread's own-cell populations, decoded to FP32 in
//    stage M(p), wait in tensor memory for the collision X(p) one plane
//    later (two plane buffers of 38 columns per warp in its 32-lane quarter,
//    tcgen05.st / tcgen05.ld); the collision issues no global loads and the
//    register file does not carry the populations through the stencil
//    stages.  At 8 rows the loads back are issued before stage F.
//  * Packed FP32: both components travel as (A, B) pairs through the moment
//    sums and the collision (two FP32 lanes per instruction).
//  * The instance descriptors travel in the kernel parameter space (up to
//    64 instances per launch): scalars and pointers come from the constant
//    bank instead of per-use global loads.
#pragma once

#include <cstring>

#include "lbfe_internal.cuh"

namespace lbfe {

typedef unsigned int u32;

// ---------------------------------------------------------------- descriptors
constexpr int kStepMaxInst = 64;

// Per-instance descriptor of one launch (kernel parameter space).
struct StepInst {
    const StepMaps *maps;          // TMA maps of fin, Cin and dens_in in global memory (when tma)
    const void *fin;               // populations read (state t)
    void *fout;                    // populations written (state t + 1)
    const float *Cin;
    float *Cout;
    const float2 *dens_in;         // offsets of the state read (reduced forms with tracking, else null)
    float2 *dens_out;              // offsets of the state written
    unsigned *status;              // per-instance status word (may be null)
    unsigned *step_ctr;            // time steps taken, two words by parity (BF16 rounding seed; may be null)
    float G, Uw, nu_A, nu_B, pi_coef, L2, inv_tauP, gx, gy, gz, rho0A, rho0B;
    u32 S, LxLy;                   // field stride, cells per plane
    unsigned short Lx, Ly, Lz, ntx, nty, zc;
    signed char visc_comp;         // 0 (A), 1 (B), -1 Newtonian
    signed char tma;               // populations (and C) by TMA
    unsigned char parity;          // ping-pong parity of the state read: step_ctr[parity] is this step's count
};
static_assert(sizeof(StepInst) <= 144, "compact launch descriptor");

// One launch covers up to kStepMaxInst instances.  A single instance takes
// the same kernel as a batch, so that batching never changes the arithmetic
// (the results of an instance are bitwise the same alone or in a batch).
struct StepArgs {
    int n, total_items;
    unsigned *status;              // status word of the launch
    unsigned *work;                // [0] work-item counter, [1] finished blocks; zero between launches
    int item_off[kStepMaxInst + 1];  // first work item of each instance
    StepInst inst[kStepMaxInst];
};

// Kernel launchers (one launch over the instances of one StepArgs).
cudaError_t step_cell_launch(const StepArgs &a, int grid, int tile_y, int precision, int advection,
                             cudaStream_t st);
cudaError_t step_cell_prepare(int tile_y, int precision, int advection, int *blocks_per_sm);
cudaError_t step_pair_launch(const StepArgs &a, int grid, int precision, cudaStream_t st);
cudaError_t step_pair_prepare(int precision, int *blocks_per_sm);

namespace {


template <int TY>
struct Geom {
    static constexpr int TX = 32;
    static constexpr int NT = TX * TY;                 // threads = tile cells
    static constexpr int WARPS = NT / 32;
    static constexpr int RX = TX + 4, RY = TY + 4;     // radius-2 region
    static constexpr int R2N = RX * RY;
    static constexpr int NRING1 = 2 * (RX - 2) + 2 * TY;  // radius-1 cells outside the tile
    static constexpr int NRING2 = 4 * TX + 4 * RY;        // radius-2 region cells outside the tile
    static constexpr int MH = (NRING2 + NT - 1) / NT;     // stage-M halo rounds per thread
    // rings: rho (float2) x3, stress scalars (a f, a) x3, j 3x2, C 6x4, u 3x3
    static constexpr int FLOATS = (2 * 3 + 2 * 3 + 6 + 24 + 9) * R2N;
    // TMEM: per warp two plane buffers in 64-column slots; warps w, w+4, ...
    // share the lane quarter w % 4 and take consecutive 128-column ranges
    // (allocations are powers of two)
    static constexpr int TMEM_USED = (WARPS / 4) * 128;
    static constexpr int TMEM_COLS = TMEM_USED <= 128 ? 128 : (TMEM_USED <= 256 ? 256 : 512);
    static_assert(WARPS % 4 == 0 && TMEM_COLS >= 32 && TMEM_COLS <= 512, "TMEM layout");
};

__device__ __forceinline__ void raise_step_flag(unsigned *global, const StepInst &I, unsigned flag) {
    atomicOr(global, flag);
    if (I.status) atomicOr(I.status, flag);
}

// ---------------------------------------------------------------- TMEM access
__device__ __forceinline__ u32 smem_addr(const void *p) { return (u32)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tm_alloc(u32 *dst, u32 ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tm_dealloc(u32 taddr, u32 ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tm_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tm_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// ---------------------------------------------------------------- TMA + mbarrier
// A wait on a copy expires after kWaitNs of GPU time (%globaltimer, read
// every 256 rounds) or kWaitRounds try_wait rounds, whichever comes first.
constexpr unsigned long long kWaitNs = 1000000000ull;
constexpr u32 kWaitRounds = 1u << 24;

__device__ __forceinline__ void mbar_init(u32 bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_init_count(u32 bar, u32 count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Arrive (release) without a byte count.
__device__ __forceinline__ void mbar_arrive(u32 bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// One thread: arm the barrier for the bytes of the copies that follow.
__device__ __forceinline__ void mbar_expect(u32 bar, u32 bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// One thread: start the copy of the box at (x, y, z, 0) into shared memory at
// dst, completing on the barrier.  x may be negative (out-of-range elements
// read as zero) but x * element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_box3(const CUtensorMap *map, u32 dst, u32 bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_box4(const CUtensorMap *map, u32 dst, u32 bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(0), "r"(bar)
        : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Predicated forms (go = 0: nothing is issued), so that the issuing code
// takes the same path whether or not a copy goes out.
__device__ __forceinline__ void mbar_expect_p(u32 bar, u32 bytes, u32 go) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t"
        "@p mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n\t}" ::"r"(bar),
        "r"(bytes), "r"(go)
        : "memory");
}
__device__ __forceinline__ void tma_box3_p(const CUtensorMap *map, u32 dst, u32 bar, int x, int y, int z, u32 go) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %6, 0;\n\t"
        "@p cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];\n\t}" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(bar), "r"(go)
        : "memory");
}
__device__ __forceinline__ void tma_box4_p(const CUtensorMap *map, u32 dst, u32 bar, int x, int y, int z, u32 go) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %7, 0;\n\t"
        "@p cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];\n\t}" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(0), "r"(bar), "r"(go)
        : "memory");
}
// Wait for the completion of phase `parity`; false once the limit expired.
__device__ __forceinline__ bool mbar_wait(u32 bar, u32 parity) {
    unsigned long long t0 = 0;
    for (u32 it = 0; it < kWaitRounds; ++it) {
        u32 ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 255u) == 255u) {
            const unsigned long long now = global_ns();
            if (t0 == 0)
                t0 = now;
            else if (now - t0 > kWaitNs)
                return false;
        }
    }
    return false;
}

__device__ __forceinline__ void tm_st32(u32 taddr, const float *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};"
                 :: "r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
                 "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
                 "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
                 "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15])),
                 "r"(__float_as_uint(v[16])), "r"(__float_as_uint(v[17])), "r"(__float_as_uint(v[18])), "r"(__float_as_uint(v[19])),
                 "r"(__float_as_uint(v[20])), "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])), "r"(__float_as_uint(v[23])),
                 "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])), "r"(__float_as_uint(v[26])), "r"(__float_as_uint(v[27])),
                 "r"(__float_as_uint(v[28])), "r"(__float_as_uint(v[29])), "r"(__float_as_uint(v[30])), "r"(__float_as_uint(v[31]))
                 );
}
__device__ __forceinline__ void tm_st4(u32 taddr, const float *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};"
                 :: "r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3]))
                 );
}
__device__ __forceinline__ void tm_st2(u32 taddr, const float *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};"
                 :: "r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1]))
                 );
}
__device__ __forceinline__ void tm_ld32(u32 taddr, u32 *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                 : 
                   "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                   "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
}
__device__ __forceinline__ void tm_ld4(u32 taddr, u32 *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
}
__device__ __forceinline__ void tm_ld2(u32 taddr, u32 *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];"
                 : "=r"(r[0]), "=r"(r[1])
                 : "r"(taddr));
}
// Completes the loads above; the registers pass through the statement so
// that no use of them can be scheduled before the wait.
__device__ __forceinline__ void tm_wait_ld38(u32 *r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 :
                 "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]),
                 "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
                 "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31]),
                 "+r"(r[32]), "+r"(r[33]), "+r"(r[34]), "+r"(r[35]), "+r"(r[36]), "+r"(r[37])
                 );
}

// The 38 populations of a cell: columns [0, 38) of a plane buffer, in the
// order (A_0, B_0, A_1, B_1, ...).
__device__ __forceinline__ void tm_store38(u32 taddr, const float *v) {
    tm_st32(taddr, v);
    tm_st4(taddr + 32, v + 32);
    tm_st2(taddr + 36, v + 36);
}
__device__ __forceinline__ void tm_load38(u32 taddr, float *v) {
    u32 r[38];
    tm_wait_st();
    tm_ld32(taddr, r);
    tm_ld4(taddr + 32, r + 32);
    tm_ld2(taddr + 36, r + 36);
    tm_wait_ld38(r);
#pragma unroll
    for (int i = 0; i < 38; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------- rings
// Ring slot of plane p (p >= -4) in rings of 2, 3 and 4 planes.
__device__ __forceinline__ int ring2(int p) { return (p + 12) & 1; }
__device__ __forceinline__ int ring3(int p) { return (p + 12) % 3; }
__device__ __forceinline__ int ring4(int p) { return (p + 12) & 3; }
__device__ __forceinline__ int wrapg(int a, int L) { a %= L; return a < 0 ? a + L : a; }

// symmetric-tensor slot of (a, b): xx, yy, zz, xy, xz, yz
__host__ __device__ constexpr int symk(int a, int b) {
    return a == b ? a : ((a + b) == 1 ? 3 : ((a + b) == 2 ? 4 : 5));
}

// Cell h (0 <= h < NRING1) of the radius-1 region outside the tile.
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

// Cell h (0 <= h < NRING2) of the radius-2 region outside the tile: first
// the four halo rows over the tile's own 32 columns (one aligned row per
// warp), then the two-column strips left and right of the tile, row by row.
template <int TY>
__device__ __forceinline__ void ring2_coord(int h, int &gx, int &gy) {
    if (h < 128) {
        const int r = h >> 5;
        gy = r < 2 ? r : TY + r;   // rows 0, 1, TY + 2, TY + 3
        gx = 2 + (h & 31);
    } else {
        const int j = h - 128;
        gy = j >> 2;               // 0 .. TY + 3
        const int c = j & 3;
        gx = c < 2 ? c : 32 + c;   // columns 0, 1, 34, 35
    }
}

extern __shared__ float4 lbfe_smem4[];
__device__ __forceinline__ float *smem() { return reinterpret_cast<float *>(lbfe_smem4); }

// Shared-memory rings (offsets in floats from the dynamic shared base).
// Values read together sit in pairs, so that one 8-byte access serves two:
//   rho  float2 [3][R2N]          (rho_A, rho_B)
//   pi   float2 [3][R2N]          (a f, a) of Pi = a (f C) - a I, a = (eta_P/tau_P) chi
//   j    [2] x (float2 [R2N] (j_x, j_y), float [R2N] j_z)          momentum
//   c    [4] x float2 [3][R2N]: (xx, xy), (yy, yz), (xz, zz)       conformation
//   u    [3] x (float2 [R2N] (u_x, u_y), float [R2N] u_z)          velocity
// (the pairs of C give each axis of the divergence and of the upwind
// stencil its three components in two 8-byte reads).  R2N is a multiple of
// 4, so every array starts on a 16-byte boundary.
template <int TY>
struct Ring {
    static constexpr int R2N = Geom<TY>::R2N;
    static_assert(R2N % 4 == 0, "ring alignment");
    static constexpr int RHO = 0, PI = 6 * R2N, J = PI + 6 * R2N, C = J + 6 * R2N, U = C + 24 * R2N;
    __device__ static float2 *rho(int s) { return reinterpret_cast<float2 *>(smem() + RHO) + s * R2N; }
    __device__ static float2 *pi(int s) { return reinterpret_cast<float2 *>(smem() + PI) + s * R2N; }
    __device__ static float2 *jxy(int s) { return reinterpret_cast<float2 *>(smem() + J + s * 3 * R2N); }
    __device__ static float *jz(int s) { return smem() + J + s * 3 * R2N + 2 * R2N; }
    // pair k (0: (xx, xy), 1: (yy, yz), 2: (xz, zz)) of C slot s
    __device__ static float2 *c(int s, int k) { return reinterpret_cast<float2 *>(smem() + C + (s * 3 + k) * 2 * R2N); }
    __device__ static float2 *uxy(int s) { return reinterpret_cast<float2 *>(smem() + U + s * 3 * R2N); }
    __device__ static float *uz(int s) { return smem() + U + s * 3 * R2N + 2 * R2N; }
};

// TMA staging of one plane.  TY = 16: the tile's own populations (box
// 32 x 16 x 38).  TY <= 12: the whole radius-2 region, populations in a box
// BW x (TY + 4) x 38 starting XPAD cells left of the tile (XPAD = 16 bytes
// of elements, so that the start is 16-byte aligned) and the conformation in
// a box 40 x (TY + 4) x 6 starting 4 cells left; region cell (gx, gy) sits
// at staging column gx - 2 + XPAD (populations), gx + 2 (C), row gy.
template <typename T, int TY>
struct Stage {
    static constexpr bool REGION = TY <= 12;
    static constexpr int XPAD = 16 / (int)sizeof(T);
    static constexpr int BW = REGION ? 32 + 2 * XPAD : 32;
    static constexpr int BH = REGION ? TY + 4 : TY;
    static constexpr int POP_PLANE = BW * BH;           // elements between populations
    static constexpr u32 POP_BYTES = (u32)(POP_PLANE * 2 * Q * sizeof(T));
    static constexpr u32 C_OFF = (POP_BYTES + 127u) & ~127u;
    static constexpr int C_PLANE = 40 * BH;              // floats between components
    static constexpr u32 C_BYTES = REGION ? (u32)(C_PLANE * 6 * sizeof(float)) : 0u;
    // offset densities of the reduced forms, 36 x BH float2 from 2 cells left
    static constexpr bool DENS = REGION && sizeof(T) == 2;
    static constexpr u32 D_OFF = (C_OFF + C_BYTES + 127u) & ~127u;
    static constexpr u32 D_BYTES = DENS ? (u32)(36 * BH * sizeof(float2)) : 0u;
    // one staging buffer (a second one, copies two planes ahead, fits 8-row
    // tiles with 2-byte storage but measured slower: 8.3 vs 9.2 G lattice
    // updates/s on 192 x 96 x 80)
    static constexpr u32 BYTES = (D_OFF + D_BYTES + 127u) & ~127u;
};


// Packed FP32 (two lanes per instruction).
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 bc(float s) { return make_float2(s, s); }

// Stage M inputs of one cell: its populations as (component A, component B)
// pairs (decoded to FP32) and 6 conformation components.  The pairs feed
// packed FP32 arithmetic (two lanes per instruction) in stages M and X.
struct MCell {
    float2 ab[Q];
    float c[6];
};

// Storage offsets (rho0_A, rho0_B) of cell n for the reduced forms.
template <typename T>
__device__ __forceinline__ float2 cell_offsets(const StepInst &I, u32 n) {
    if (!Store<T>::offset) return make_float2(0.f, 0.f);
    if (I.dens_in) return __ldcg(I.dens_in + n);
    return make_float2(I.rho0A, I.rho0B);
}

// Cell offsets are 32-bit: an instance holds at most 2^26 cells, so every
// field offset (s*19 + i)*S + n stays below 2^32.
template <typename T>
__device__ __forceinline__ void m_load(const StepInst &I, const T *__restrict__ fin, const float *__restrict__ Cin,
                                       u32 S, u32 n, MCell &m) {
    const float2 o = cell_offsets<T>(I, n);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        m.ab[i].x = Store<T>::ld_l2(fin + (u32)(i * S + n));
        m.ab[i].y = Store<T>::ld_l2(fin + (u32)((Q + i) * S + n));
        if (Store<T>::offset) m.ab[i] = fma2(bc(wq(i)), o, m.ab[i]);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) m.c[k] = __ldcg(Cin + (u32)(k * S + n));
}

// As m_load, with the populations taken from the TMA staging buffer
// (element (x, y, i) of the box at i * NT + y * 32 + x).
template <typename T, int NT>
__device__ __forceinline__ void m_load_staged(const StepInst &I, const T *stage, int t,
                                              const float *__restrict__ Cin, u32 S, u32 n, MCell &m) {
    const float2 o = cell_offsets<T>(I, n);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        m.ab[i].x = Store<T>::ld_plain(stage + i * NT + t);
        m.ab[i].y = Store<T>::ld_plain(stage + (Q + i) * NT + t);
        if (Store<T>::offset) m.ab[i] = fma2(bc(wq(i)), o, m.ab[i]);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) m.c[k] = __ldg(Cin + (u32)(k * S + n));
}

// As m_load, for region cell (gx, gy) staged by a region copy (Stage).
template <typename T, int TY>
__device__ __forceinline__ void m_load_region(const StepInst &I, const T *sp, const float *sc, int gx, int gy, u32 n,
                                              MCell &m) {
    using St = Stage<T, TY>;
    // offset densities: staged with the region when tracked per cell
    float2 o = make_float2(0.f, 0.f);
    if (Store<T>::offset) {
        if (St::DENS && I.dens_in)
            o = reinterpret_cast<const float2 *>(reinterpret_cast<const char *>(sp) + St::D_OFF)[gy * 36 + gx];
        else
            o = cell_offsets<T>(I, n);
    }
    const int e = gy * St::BW + gx - 2 + St::XPAD;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        m.ab[i].x = Store<T>::ld_plain(sp + i * St::POP_PLANE + e);
        m.ab[i].y = Store<T>::ld_plain(sp + (Q + i) * St::POP_PLANE + e);
        if (Store<T>::offset) m.ab[i] = fma2(bc(wq(i)), o, m.ab[i]);
    }
    const int ec = gy * 40 + gx + 2;
#pragma unroll
    for (int k = 0; k < 6; ++k) m.c[k] = sc[k * St::C_PLANE + ec];
}

// Stage M for one cell: moments, stress scalars and conformation into the
// ring slots of its plane.  Both components' sums run as packed pairs; the
// momentum is summed from opposite-pair differences f_i - f_opp(i) (exact
// in FP32 per pair), per component, and the components added at the end.
template <int TY>
__device__ __forceinline__ void m_store(const StepInst &I, const MCell &m, int idx, int s3, int s2, int s4) {
    // s3: rho / stress slot, s2: j slot, s4: C slot of the plane
    using Rg = Ring<TY>;
    float2 r = m.ab[0];
#pragma unroll
    for (int i = 1; i < Q; ++i) r = add2(r, m.ab[i]);
    float2 jx = bc(0.f), jy = jx, jz = jx;
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const float2 d = sub2(m.ab[i], m.ab[i + 1]);
        if (cx(i)) jx = cx(i) > 0 ? add2(jx, d) : sub2(jx, d);
        if (cy(i)) jy = cy(i) > 0 ? add2(jy, d) : sub2(jy, d);
        if (cz(i)) jz = cz(i) > 0 ? add2(jz, d) : sub2(jz, d);
    }
    Rg::rho(s3)[idx] = r;
    Rg::jxy(s2)[idx] = make_float2(jx.x + jx.y, jy.x + jy.y);
    Rg::jz(s2)[idx] = jz.x + jz.y;
    // C components xx, yy, zz, xy, xz, yz = m.c[0..5]
    Rg::c(s4, 0)[idx] = make_float2(m.c[0], m.c[3]);
    Rg::c(s4, 1)[idx] = make_float2(m.c[1], m.c[5]);
    Rg::c(s4, 2)[idx] = make_float2(m.c[4], m.c[2]);
    float a = 0.f, fp = 1.f;
    if (I.visc_comp >= 0) {
        a = I.pi_coef * (I.visc_comp == 0 ? r.x : r.y) / (r.x + r.y);
        fp = peterlin(I.L2, m.c[0], m.c[1], m.c[2]);
    }
    Rg::pi(s3)[idx] = make_float2(a * fp, a);
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
__device__ __forceinline__ void stage_f_cell(const StepInst &I, int idx, const Slots &L, float FA[3], float FB[3],
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
        const float2 *pc = Rg::pi(L.r3[1]);
        const float2 Ax = pc[idx + 1], Bx = pc[idx - 1], Ay = pc[idx + RX], By = pc[idx - RX];
        const float2 Az = Rg::pi(L.r3[2])[idx], Bz = Rg::pi(L.r3[0])[idx];
        // x-neighbours: C_xx, C_xy (pair 0), C_xz (pair 2)
        const float2 *c0 = Rg::c(L.cf[1], 0), *c1 = Rg::c(L.cf[1], 1), *c2 = Rg::c(L.cf[1], 2);
        const float2 xp0 = c0[idx + 1], xm0 = c0[idx - 1];
        const float xp2 = c2[idx + 1].x, xm2 = c2[idx - 1].x;
        // y-neighbours: C_xy (pair 0), C_yy, C_yz (pair 1)
        const float yp0 = c0[idx + RX].y, ym0 = c0[idx - RX].y;
        const float2 yp1 = c1[idx + RX], ym1 = c1[idx - RX];
        // z-neighbours (planes q + 1, q - 1): C_xz, C_zz (pair 2), C_yz (pair 1)
        const float2 zp2 = Rg::c(L.cf[2], 2)[idx], zm2 = Rg::c(L.cf[0], 2)[idx];
        const float zp1 = Rg::c(L.cf[2], 1)[idx].y, zm1 = Rg::c(L.cf[0], 1)[idx].y;
        // a = x
        float gxd = Ax.x * xp0.x - Bx.x * xm0.x;
        float gyd = Ay.x * yp0 - By.x * ym0;
        float gzd = Az.x * zp2.x - Bz.x * zm2.x;
        gxd -= Ax.y - Bx.y;
        FP[0] = 0.5f * (gxd + gyd + gzd);
        // a = y
        gxd = Ax.x * xp0.y - Bx.x * xm0.y;
        gyd = Ay.x * yp1.x - By.x * ym1.x;
        gzd = Az.x * zp1 - Bz.x * zm1;
        gyd -= Ay.y - By.y;
        FP[1] = 0.5f * (gxd + gyd + gzd);
        // a = z
        gxd = Ax.x * xp2 - Bx.x * xm2;
        gyd = Ay.x * yp1.y - By.x * ym1.y;
        gzd = Az.x * zp2.y - Bz.x * zm2.y;
        gzd -= Az.y - Bz.y;
        FP[2] = 0.5f * (gxd + gyd + gzd);
    }
    const float g[3] = {I.gx, I.gy, I.gz};
    const float inv = 1.0f / (rA + rB);
    const float2 jxy = Rg::jxy(L.j3)[idx];
    const float j[3] = {jxy.x, jxy.y, Rg::jz(L.j3)[idx]};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        FA[a] = -I.G * rA * sA[a] + (rA * inv) * FP[a] + rA * g[a];
        FB[a] = -I.G * rB * sB[a] + (rB * inv) * FP[a] + rB * g[a];
        u[a] = (j[a] + 0.5f * (FA[a] + FB[a])) * inv;
    }
    Rg::uxy(L.r3[1])[idx] = make_float2(u[0], u[1]);
    Rg::uz(L.r3[1])[idx] = u[2];
}

__device__ __forceinline__ float minmodf(float a, float b) {
    if (a * b <= 0.f) return 0.f;
    return fabsf(a) < fabsf(b) ? a : b;
}

// Stage U for one cell (ring index idx) of plane r: the FENE-P update of
// Eq. 2 (Eq. 4) with central grad u (u_ghost = 2 U_wall - u at the walls)
// and first-order upwind u . grad C (C mirrored at the walls).  Writes the
// new conformation to cn; returns false when tr C reached L^2.
// ADV2: u . grad C by the second-order minmod-limited upwind scheme instead
// of the first-order one.  Along an axis with speed |v|, upwind neighbour a,
// the next one aa and the downwind neighbour b, the contribution is
//   |v| [(c - a) + (minmod(b - c, c - a) - minmod(c - a, a - aa)) / 2],
// the difference of the two face values reconstructed from the upwind side
// (the same for either sign of v).  z needs C of plane r - 2, which the ring
// no longer holds: cprev carries the cell's own C of that plane from the
// previous call (and is updated to plane r - 1 here).
template <int TY, bool ADV2 = false>
__device__ __forceinline__ bool stage_u_cell(const StepInst &I, int idx, const Slots &L, int r, float cn[6],
                                             float *cprev = nullptr) {
    constexpr int RX = Geom<TY>::RX;
    using Rg = Ring<TY>;
    const float Uw = I.Uw;
    const int Lz = I.Lz;
    const float2 *uxc = Rg::uxy(L.ur[1]);
    const float *uzc = Rg::uz(L.ur[1]);
    const float2 u01 = uxc[idx];
    const float u0[3] = {u01.x, u01.y, uzc[idx]};
    // neighbours of plane r along x and y, and of the own column in z
    const float2 axp = uxc[idx + 1], axm = uxc[idx - 1], ayp = uxc[idx + RX], aym = uxc[idx - RX];
    const float zxp = uzc[idx + 1], zxm = uzc[idx - 1], zyp = uzc[idx + RX], zym = uzc[idx - RX];
    const float2 up01 = Rg::uxy(L.ur[2])[idx], um01 = Rg::uxy(L.ur[0])[idx];
    const float upn[3] = {up01.x, up01.y, Rg::uz(L.ur[2])[idx]};
    const float umn[3] = {um01.x, um01.y, Rg::uz(L.ur[0])[idx]};
    const float uxp[3] = {axp.x, axp.y, zxp}, uxm[3] = {axm.x, axm.y, zxm};
    const float uyp[3] = {ayp.x, ayp.y, zyp}, uym[3] = {aym.x, aym.y, zym};
    float Gr[3][3];
    // grad u by central differences, u_ghost = 2 U_wall - u at the walls
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float uwb = j == 0 ? -Uw : 0.f, uwt = j == 0 ? Uw : 0.f;
        const float uzp = (r == Lz - 1) ? 2.f * uwt - u0[j] : upn[j];
        const float uzm = (r == 0) ? 2.f * uwb - u0[j] : umn[j];
        Gr[0][j] = 0.5f * (uxp[j] - uxm[j]);
        Gr[1][j] = 0.5f * (uyp[j] - uym[j]);
        Gr[2][j] = 0.5f * (uzp - uzm);
    }
    // C components xx, yy, zz, xy, xz, yz from the pairs (xx, xy), (yy, yz), (xz, zz)
    auto c_at = [&](int s, int n, float out[6]) {
        const float2 p0 = Rg::c(s, 0)[n], p1 = Rg::c(s, 1)[n], p2 = Rg::c(s, 2)[n];
        out[0] = p0.x; out[1] = p1.x; out[2] = p2.y; out[3] = p0.y; out[4] = p2.x; out[5] = p1.y;
    };
    float c[6];
    c_at(L.cu[1], idx, c);
    // upwind u . grad C (C mirrored at the walls)
    const int ox = u0[0] > 0.f ? -1 : 1, oy = u0[1] > 0.f ? -RX : RX;
    const float sx = u0[0] > 0.f ? u0[0] : -u0[0], sy = u0[1] > 0.f ? u0[1] : -u0[1];
    const float sz = u0[2] > 0.f ? u0[2] : -u0[2];
    float adv[6];
    if constexpr (!ADV2) {
        float cx_[6], cy_[6], cz6[6];
        c_at(L.cu[1], idx + ox, cx_);
        c_at(L.cu[1], idx + oy, cy_);
        c_at(u0[2] > 0.f ? L.cu[0] : L.cu[2], idx, cz6);
#pragma unroll
        for (int q6 = 0; q6 < 6; ++q6)
            adv[q6] = sx * (c[q6] - cx_[q6]) + sy * (c[q6] - cy_[q6]) + sz * (c[q6] - cz6[q6]);
    } else {
        float xa[6], xaa[6], xb[6], ya[6], yaa[6], yb[6], zm1[6], zp1[6], zp2[6];
        c_at(L.cu[1], idx + ox, xa);
        c_at(L.cu[1], idx + 2 * ox, xaa);
        c_at(L.cu[1], idx - ox, xb);
        c_at(L.cu[1], idx + oy, ya);
        c_at(L.cu[1], idx + 2 * oy, yaa);
        c_at(L.cu[1], idx - oy, yb);
        c_at(L.cu[0], idx, zm1);    // plane r - 1
        c_at(L.cu[2], idx, zp1);    // plane r + 1
        c_at(L.cf[2], idx, zp2);    // plane r + 2
        const bool zup = u0[2] > 0.f;
        auto lim = [](float c0, float a, float aa, float b) {
            return (c0 - a) + 0.5f * (minmodf(b - c0, c0 - a) - minmodf(c0 - a, a - aa));
        };
#pragma unroll
        for (int q6 = 0; q6 < 6; ++q6) {
            const float za = zup ? zm1[q6] : zp1[q6], zaa = zup ? cprev[q6] : zp2[q6], zb = zup ? zp1[q6] : zm1[q6];
            adv[q6] = sx * lim(c[q6], xa[q6], xaa[q6], xb[q6]) + sy * lim(c[q6], ya[q6], yaa[q6], yb[q6]) +
                      sz * lim(c[q6], za, zaa, zb);
        }
#pragma unroll
        for (int q6 = 0; q6 < 6; ++q6) cprev[q6] = zm1[q6];
    }
    const float Cm[3][3] = {{c[0], c[3], c[4]}, {c[3], c[1], c[5]}, {c[4], c[5], c[2]}};
    const float fp = peterlin(I.L2, c[0], c[1], c[2]);
#pragma unroll
    for (int q6 = 0; q6 < 6; ++q6) {
        const int a = q6 < 3 ? q6 : (q6 == 5 ? 1 : 0);
        const int b = q6 < 3 ? q6 : (q6 == 3 ? 1 : 2);
        float st = 0.f;
#pragma unroll
        for (int m = 0; m < 3; ++m) st += Cm[a][m] * Gr[m][b] + Gr[m][a] * Cm[m][b];
        const float relax = (fp * c[q6] - (q6 < 3 ? 1.f : 0.f)) * I.inv_tauP;
        cn[q6] = c[q6] + (-adv[q6] + st - relax);
    }
    return c[0] + c[1] + c[2] < I.L2;
}

// Offsets of the reduced storage forms at the destination of a push:
// the destination cell's densities (rho_A, rho_B) of this step (from the
// density ring of planes q-1, q, q+1), or the constant offsets when
// densities are not tracked.
struct PushOffsets {
    const float2 *ring[3];   // density ring slots of planes q-1, q, q+1
    int idx;                 // ring index of the pushing cell
    float2 own;              // the pushing cell's densities
    bool track;
    float2 r0;               // constant offsets
    unsigned seed;           // the instance's step count (stochastic rounding)
};

template <int RX>
__device__ __forceinline__ float2 push_offset(const PushOffsets &P, int d, bool wall) {
    if (!P.track) return P.r0;
    if (wall) return P.own;
    return P.ring[cz(d) + 1][P.idx + cx(d) + cy(d) * RX];
}

// Store post-collision population d of both components (lanes x: A, y: B)
// of the cell at offset n into its streamed position x + c_d.  With WALLS,
// a population whose target lies beyond a wall returns into the cell as the
// opposite direction (halfway bounce-back) with the moving-wall term
// -6 w_d rho_s (c_d . U_wall).
template <typename T, bool WALLS, int RX>
__device__ __forceinline__ void push_ab(T *__restrict__ fdst, u32 S, int d, float2 v, float2 rs,
                                        const PushOffsets &P, u32 n, bool bottom, bool top, float Uw, int LxLy,
                                        const int dxy[3][3]) {
    int dir = d;
    u32 dst = n + (u32)(cz(d) * LxLy + dxy[cx(d) + 1][cy(d) + 1]);
    bool wall = false;
    if (WALLS && ((cz(d) < 0 && bottom) || (cz(d) > 0 && top))) {
        v = fma2(bc(-6.f * wq(d) * (float)cx(d) * (cz(d) < 0 ? -Uw : Uw)), rs, v);
        dir = opp(d);
        dst = n;
        wall = true;
    }
    if (Store<T>::offset) v = fma2(bc(-wq(d)), push_offset<RX>(P, d, wall), v);
    const unsigned r = Store<T>::sround ? sround_bits(dst, dir, P.seed) : 0u;
    Store<T>::st_sr(fdst + (u32)(dir * S + dst), v.x, r);
    Store<T>::st_sr(fdst + (u32)((Q + dir) * S + dst), v.y, r >> 16);
}

// BGK + Guo collision of both components of one cell, on packed FP32 (lane
// x: component A, lane y: component B), and push streaming.  Opposite
// directions share the symmetric parts:
//   f^eq_{i,-i} = w rho (1 + 9/2 (c.u)^2 - 3/2 u.u) +- 3 w rho (c.u)
//   S_{i,-i}    = (1 - 1/2tau) w (9 (c.u)(c.F) - 3 u.F) +- 3 (1 - 1/2tau) w (c.F)
// so that with E = omega rho (1 - 3/2 u.u) - 3 (1 - 1/2tau) u.F the
// post-collision pair is (1 - omega) f_{i,-i} + sym +- anti,
//   sym  = w E + (c.u) (9/2 omega rho w (c.u) + 9 (1 - 1/2tau) w (c.F)),
//   anti = 3 omega rho w (c.u) + 3 (1 - 1/2tau) w (c.F),
// with the weight products formed once per weight class.  u and omega are
// common to both components; rho and F are per component.
template <typename T, bool WALLS, int RX>
__device__ __forceinline__ void collide_push_ab(const float2 *fv, T *__restrict__ fdst, u32 S, float2 rs,
                                                const PushOffsets &P, const float u[3], const float2 F[3], float om,
                                                u32 n, bool bottom, bool top, float Uw, int LxLy,
                                                const int dxy[3][3]) {
    const float omc = 1.0f - om, pref = 1.0f - 0.5f * om;
    const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const float2 u2[3] = {bc(u[0]), bc(u[1]), bc(u[2])};
    const float2 uF = fma2(u2[2], F[2], fma2(u2[1], F[1], mul2(u2[0], F[0])));
    const float2 E = fma2(bc(-3.f * pref), uF, mul2(bc(om * (1.f - 1.5f * uu)), rs));
    const float2 omc2 = bc(omc);
    {
        float2 v = fma2(omc2, fv[0], mul2(bc(wq(0)), E));
        if (Store<T>::offset) v = fma2(bc(-wq(0)), P.track ? P.own : P.r0, v);
        const unsigned r = Store<T>::sround ? sround_bits(n, 0, P.seed) : 0u;
        Store<T>::st_sr(fdst + n, v.x, r);
        Store<T>::st_sr(fdst + (u32)(Q * S + n), v.y, r >> 16);
    }
    // weight classes: faces (i = 1..6) and edges (i = 7..18)
    float2 Ew[2], a1w[2], b1w[2], a2w[2], b2w[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const float w = wq(c == 0 ? 1 : 7);
        Ew[c] = mul2(bc(w), E);
        a1w[c] = mul2(bc(4.5f * om * w), rs);
        b1w[c] = bc(9.f * pref * w);
        a2w[c] = mul2(bc(3.f * om * w), rs);
        b2w[c] = bc(3.f * pref * w);
    }
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const int c = i <= 6 ? 0 : 1;
        float2 cu = bc(0.f), cF = cu;
        bool first = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int ca = a == 0 ? cx(i) : (a == 1 ? cy(i) : cz(i));
            if (!ca) continue;
            if (first) {
                cu = ca > 0 ? u2[a] : mul2(bc(-1.f), u2[a]);
                cF = ca > 0 ? F[a] : mul2(bc(-1.f), F[a]);
                first = false;
            } else {
                cu = ca > 0 ? add2(cu, u2[a]) : sub2(cu, u2[a]);
                cF = ca > 0 ? add2(cF, F[a]) : sub2(cF, F[a]);
            }
        }
        const float2 sym = fma2(cu, fma2(a1w[c], cu, mul2(b1w[c], cF)), Ew[c]);
        const float2 anti = fma2(a2w[c], cu, mul2(b2w[c], cF));
        push_ab<T, WALLS, RX>(fdst, S, i, fma2(omc2, fv[i], add2(sym, anti)), rs, P, n, bottom, top, Uw, LxLy, dxy);
        push_ab<T, WALLS, RX>(fdst, S, i + 1, fma2(omc2, fv[i + 1], sub2(sym, anti)), rs, P, n, bottom, top, Uw,
                              LxLy, dxy);
    }
}

// Called by every block once it has taken its last item: the last block to
// finish returns the two counters to zero for the next launch (no other
// block reads them any more).  The fence orders the block's last fetch on
// work[0] before its arrival on work[1], so the last arriver's reset comes
// after every other block's final fetch; the reset itself is atomic and
// fenced before the kernel ends.
__device__ __forceinline__ void release_work_counters(unsigned *work) {
    __threadfence();
    if (atomicAdd(work + 1, 1u) == gridDim.x - 1) {
        __threadfence();
        atomicExch(work, 0u);
        atomicExch(work + 1, 0u);
        __threadfence();
    }
}

// The step count that seeds the BF16 stochastic rounding of instance k's
// stores in this launch: step_ctr[parity].  The block that takes the
// instance's first work item also writes step_ctr[parity ^ 1], the count of
// the next launch, which no block of this launch reads (so no ordering
// between the blocks is needed).  Other storage forms read nothing.
template <bool SROUND>
__device__ __forceinline__ unsigned step_seed(const StepArgs &A, const StepInst &I, int k, int item, int t) {
    if (!SROUND || !I.step_ctr) return 0u;
    const unsigned s = __ldcg(I.step_ctr + I.parity);
    if (t == 0 && item == A.item_off[k]) I.step_ctr[I.parity ^ 1] = s + 1u;
    return s;
}

// Position of work item `item`: instance, column tile and z-chunk.
struct ItemPos {
    int k, bx, by, z0, z1;
};

template <int TY>
__device__ __forceinline__ ItemPos item_pos(const StepArgs &A, int item) {
    ItemPos P;
    P.k = 0;
    for (int hi = A.n - 1; P.k < hi;) {
        const int mid = (P.k + hi + 1) >> 1;
        if (A.item_off[mid] <= item) P.k = mid; else hi = mid - 1;
    }
    const StepInst &I = A.inst[P.k];
    int local = item - A.item_off[P.k];
    P.bx = local % I.ntx;
    local /= I.ntx;
    P.by = local % I.nty;
    P.z0 = (local / I.nty) * I.zc;
    P.z1 = min(I.Lz, P.z0 + I.zc);
    return P;
}

template <typename T, int TY>
__device__ __forceinline__ void issue_plane(const StepArgs &A, const ItemPos &P, int plane, u32 dst, u32 bar,
                                            u32 go = 1u) {
    using St = Stage<T, TY>;
    const StepInst &I = A.inst[P.k];
    const int z = min(max(plane, 0), I.Lz - 1);
    if (St::REGION) {
        const bool dcopy = St::DENS && I.dens_in != nullptr;   // offset densities tracked per cell
        mbar_expect_p(bar, St::POP_BYTES + St::C_BYTES + (dcopy ? St::D_BYTES : 0u), go);
        tma_box4_p(&I.maps->pop, dst, bar, P.bx * 32 - St::XPAD, P.by * TY - 2, z, go);
        tma_box4_p(&I.maps->c, dst + St::C_OFF, bar, P.bx * 32 - 4, P.by * TY - 2, z, go);
        if (dcopy) tma_box3_p(&I.maps->dens, dst + St::D_OFF, bar, P.bx * 32 - 2, P.by * TY - 2, z, go);
    } else {
        mbar_expect_p(bar, St::POP_BYTES, go);
        tma_box4_p(&I.maps->pop, dst, bar, P.bx * 32, P.by * TY, z, go);
    }
}

}  // namespace

}  // namespace lbfe
