// lbfe_fused2.cu -- the time-step kernel with two x-adjacent cells per
// thread: tiles of 32 x 16 cells, 256 threads, thread (lx, ty) owning the
// cells x = 2 lx and 2 lx + 1 of row ty.  Same stages, rings, TMA staging
// and lags as the one-cell kernel (lbfe_step.cuh); per thread the two cells
// travel as float2 pairs:
//   * populations and conformation move as 8-byte pairs (LDG/LDS/STG.64,
//     half2 / bfloat162 for the reduced forms): half the memory instructions
//     and address arithmetic of one cell per thread;
//   * moments and the BGK + Guo collision run on packed FP32 (__fadd2_rn,
//     __fmul2_rn, __ffma2_rn: two lanes of FP32 per instruction);
//   * the 2 x 38 decoded populations wait in TMEM between stage M and the
//     collision (76 columns per thread and plane buffer).
// Pushes along +-x leave the pair (x, x+1) misaligned and are stored per
// cell; all other directions and the bounce-back into the cell itself are
// pair stores.  Needs even Lx (pairs never straddle the periodic seam).
#include "lbfe_step.cuh"

namespace lbfe {

namespace {

constexpr int PTY = 16;                       // tile rows
constexpr int PNT = 256;                      // threads
using PG = Geom<PTY>;                         // region and ring geometry of the 32 x 16 tile
constexpr int NPAIR_HALO = 4 * 18 + 2 * PTY;  // radius-2 region pairs outside the tile
constexpr int P_TMEM_COLS = 512;              // 8 warps, two per lane quarter, 256 columns each

// Pair access of two adjacent elements of one population array.
template <typename T>
struct Pair;
template <>
struct Pair<float> {
    static __device__ __forceinline__ float2 ldg(const float *p) { return __ldcg(reinterpret_cast<const float2 *>(p)); }
    static __device__ __forceinline__ float2 lds(const float *p) { return *reinterpret_cast<const float2 *>(p); }
    static __device__ __forceinline__ void stg(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
};
template <>
struct Pair<__half> {
    static __device__ __forceinline__ float2 ldg(const __half *p) {
        return __half22float2(__ldcg(reinterpret_cast<const __half2 *>(p)));
    }
    static __device__ __forceinline__ float2 lds(const __half *p) {
        return __half22float2(*reinterpret_cast<const __half2 *>(p));
    }
    static __device__ __forceinline__ void stg(__half *p, float2 v) {
        *reinterpret_cast<__half2 *>(p) = __float22half2_rn(v);
    }
};
template <>
struct Pair<__nv_bfloat16> {
    static __device__ __forceinline__ float2 ldg(const __nv_bfloat16 *p) {
        return __bfloat1622float2(__ldcg(reinterpret_cast<const __nv_bfloat162 *>(p)));
    }
    static __device__ __forceinline__ float2 lds(const __nv_bfloat16 *p) {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
    }
    static __device__ __forceinline__ void stg(__nv_bfloat16 *p, float2 v) {
        *reinterpret_cast<__nv_bfloat162 *>(p) = __float22bfloat162_rn(v);
    }
};

// ---------------------------------------------------------------- TMEM, 76 columns
__device__ __forceinline__ void tm_st64(u32 taddr, const float *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x64.b32 [%0], {"
                 "%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16,"
                 "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32,"
                 "%33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48,"
                 "%49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63, %64"
                 "};"
                 :: "r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
                 "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
                 "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
                 "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15])),
                 "r"(__float_as_uint(v[16])), "r"(__float_as_uint(v[17])), "r"(__float_as_uint(v[18])), "r"(__float_as_uint(v[19])),
                 "r"(__float_as_uint(v[20])), "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])), "r"(__float_as_uint(v[23])),
                 "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])), "r"(__float_as_uint(v[26])), "r"(__float_as_uint(v[27])),
                 "r"(__float_as_uint(v[28])), "r"(__float_as_uint(v[29])), "r"(__float_as_uint(v[30])), "r"(__float_as_uint(v[31])),
                 "r"(__float_as_uint(v[32])), "r"(__float_as_uint(v[33])), "r"(__float_as_uint(v[34])), "r"(__float_as_uint(v[35])),
                 "r"(__float_as_uint(v[36])), "r"(__float_as_uint(v[37])), "r"(__float_as_uint(v[38])), "r"(__float_as_uint(v[39])),
                 "r"(__float_as_uint(v[40])), "r"(__float_as_uint(v[41])), "r"(__float_as_uint(v[42])), "r"(__float_as_uint(v[43])),
                 "r"(__float_as_uint(v[44])), "r"(__float_as_uint(v[45])), "r"(__float_as_uint(v[46])), "r"(__float_as_uint(v[47])),
                 "r"(__float_as_uint(v[48])), "r"(__float_as_uint(v[49])), "r"(__float_as_uint(v[50])), "r"(__float_as_uint(v[51])),
                 "r"(__float_as_uint(v[52])), "r"(__float_as_uint(v[53])), "r"(__float_as_uint(v[54])), "r"(__float_as_uint(v[55])),
                 "r"(__float_as_uint(v[56])), "r"(__float_as_uint(v[57])), "r"(__float_as_uint(v[58])), "r"(__float_as_uint(v[59])),
                 "r"(__float_as_uint(v[60])), "r"(__float_as_uint(v[61])), "r"(__float_as_uint(v[62])), "r"(__float_as_uint(v[63])));
}
__device__ __forceinline__ void tm_st8(u32 taddr, const float *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                 :: "r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
                 "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])));
}
__device__ __forceinline__ void tm_ld64(u32 taddr, u32 *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x64.b32 {"
                 "%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                 "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, "
                 "%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, "
                 "%48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];"
                 :
                 "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                 "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                 "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
                 "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
                 "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
                 "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
                 "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
                 : "r"(taddr));
}
__device__ __forceinline__ void tm_ld8(u32 taddr, u32 *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {"
                 "%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 :
                 "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}
__device__ __forceinline__ void tm_wait_ld76(u32 *r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 :
                 "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]),
                 "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
                 "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31]),
                 "+r"(r[32]), "+r"(r[33]), "+r"(r[34]), "+r"(r[35]), "+r"(r[36]), "+r"(r[37]), "+r"(r[38]), "+r"(r[39]),
                 "+r"(r[40]), "+r"(r[41]), "+r"(r[42]), "+r"(r[43]), "+r"(r[44]), "+r"(r[45]), "+r"(r[46]), "+r"(r[47]),
                 "+r"(r[48]), "+r"(r[49]), "+r"(r[50]), "+r"(r[51]), "+r"(r[52]), "+r"(r[53]), "+r"(r[54]), "+r"(r[55]),
                 "+r"(r[56]), "+r"(r[57]), "+r"(r[58]), "+r"(r[59]), "+r"(r[60]), "+r"(r[61]), "+r"(r[62]), "+r"(r[63]),
                 "+r"(r[64]), "+r"(r[65]), "+r"(r[66]), "+r"(r[67]), "+r"(r[68]), "+r"(r[69]), "+r"(r[70]), "+r"(r[71]),
                 "+r"(r[72]), "+r"(r[73]), "+r"(r[74]), "+r"(r[75]));
}

// Columns 2i and 2i + 1 hold population i of the first and second cell.
__device__ __forceinline__ void tm_store76(u32 taddr, const float2 *f) {
    float v[76];
#pragma unroll
    for (int i = 0; i < 38; ++i) {
        v[2 * i] = f[i].x;
        v[2 * i + 1] = f[i].y;
    }
    tm_st64(taddr, v);
    tm_st8(taddr + 64, v + 64);
    tm_st4(taddr + 72, v + 72);
}
__device__ __forceinline__ void tm_load76(u32 taddr, float2 *f) {
    u32 r[76];
    tm_wait_st();
    tm_ld64(taddr, r);
    tm_ld8(taddr + 64, r + 64);
    tm_ld4(taddr + 72, r + 72);
    tm_wait_ld76(r);
#pragma unroll
    for (int i = 0; i < 38; ++i) f[i] = make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
}

// ---------------------------------------------------------------- stage M, pairs
struct MPair {
    float2 f[2 * Q];
    float2 c[6];
};

template <typename T>
__device__ __forceinline__ void pair_offsets(const StepInst &I, u32 n, float2 &ra0, float2 &rb0) {
    ra0 = rb0 = make_float2(0.f, 0.f);
    if (Store<T>::offset) {
        if (I.dens_in) {
            const float4 od = __ldcg(reinterpret_cast<const float4 *>(I.dens_in + n));
            ra0 = make_float2(od.x, od.z);
            rb0 = make_float2(od.y, od.w);
        } else {
            ra0 = bc(I.rho0A);
            rb0 = bc(I.rho0B);
        }
    }
}

// The pair (n, n + 1), n even, from global memory.
template <typename T>
__device__ __forceinline__ void m_load2(const StepInst &I, const T *__restrict__ fin, const float *__restrict__ Cin,
                                        u32 S, u32 n, MPair &m) {
    float2 ra0, rb0;
    pair_offsets<T>(I, n, ra0, rb0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        m.f[i] = Pair<T>::ldg(fin + (u32)(i * S + n));
        m.f[Q + i] = Pair<T>::ldg(fin + (u32)((Q + i) * S + n));
        if (Store<T>::offset) {
            m.f[i] = fma2(bc(wq(i)), ra0, m.f[i]);
            m.f[Q + i] = fma2(bc(wq(i)), rb0, m.f[Q + i]);
        }
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) m.c[k] = Pair<float>::ldg(Cin + (u32)(k * S + n));
}

// The pair from the TMA staging buffer (element (x, y, i) at i * 512 + y * 32 + x; e = y * 32 + x).
template <typename T>
__device__ __forceinline__ void m_load2_staged(const StepInst &I, const T *stage, int e,
                                               const float *__restrict__ Cin, u32 S, u32 n, MPair &m) {
    float2 ra0, rb0;
    pair_offsets<T>(I, n, ra0, rb0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        m.f[i] = Pair<T>::lds(stage + i * 512 + e);
        m.f[Q + i] = Pair<T>::lds(stage + (Q + i) * 512 + e);
        if (Store<T>::offset) {
            m.f[i] = fma2(bc(wq(i)), ra0, m.f[i]);
            m.f[Q + i] = fma2(bc(wq(i)), rb0, m.f[Q + i]);
        }
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) m.c[k] = Pair<float>::ldg(Cin + (u32)(k * S + n));
}

// Moments, stress scalars and conformation of the pair at ring index idx
// (even) into the ring slots of its plane.
__device__ __forceinline__ void m_store2(const StepInst &I, const MPair &m, int idx, int s3, int s2, int s4) {
    using Rg = Ring<PTY>;
    float2 rA = make_float2(0.f, 0.f), rB = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        rA = add2(rA, m.f[i]);
        rB = add2(rB, m.f[Q + i]);
    }
    // momentum from opposite-pair differences (exact in FP32 per pair)
    float2 jx = make_float2(0.f, 0.f), jy = jx, jz = jx;
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const float2 d = add2(sub2(m.f[i], m.f[i + 1]), sub2(m.f[Q + i], m.f[Q + i + 1]));
        if (cx(i)) jx = cx(i) > 0 ? add2(jx, d) : sub2(jx, d);
        if (cy(i)) jy = cy(i) > 0 ? add2(jy, d) : sub2(jy, d);
        if (cz(i)) jz = cz(i) > 0 ? add2(jz, d) : sub2(jz, d);
    }
    // both cells (idx even) in one 16-byte store per ring array
    *reinterpret_cast<float4 *>(Rg::rho(s3) + idx) = make_float4(rA.x, rB.x, rA.y, rB.y);
    *reinterpret_cast<float4 *>(Rg::jxy(s2) + idx) = make_float4(jx.x, jy.x, jx.y, jy.y);
    *reinterpret_cast<float2 *>(Rg::jz(s2) + idx) = jz;
    // C components xx, yy, zz, xy, xz, yz = m.c[0..5]; pairs (xx, xy), (yy, yz), (xz, zz)
    *reinterpret_cast<float4 *>(Rg::c(s4, 0) + idx) = make_float4(m.c[0].x, m.c[3].x, m.c[0].y, m.c[3].y);
    *reinterpret_cast<float4 *>(Rg::c(s4, 1) + idx) = make_float4(m.c[1].x, m.c[5].x, m.c[1].y, m.c[5].y);
    *reinterpret_cast<float4 *>(Rg::c(s4, 2) + idx) = make_float4(m.c[4].x, m.c[2].x, m.c[4].y, m.c[2].y);
    float2 af = make_float2(0.f, 0.f), a = af;
    if (I.visc_comp >= 0) {
        const float2 rv = I.visc_comp == 0 ? rA : rB;
        a.x = I.pi_coef * rv.x / (rA.x + rB.x);
        a.y = I.pi_coef * rv.y / (rA.y + rB.y);
        af.x = a.x * peterlin(I.L2, m.c[0].x, m.c[1].x, m.c[2].x);
        af.y = a.y * peterlin(I.L2, m.c[0].y, m.c[1].y, m.c[2].y);
    }
    *reinterpret_cast<float4 *>(Rg::pi(s3) + idx) = make_float4(af.x, a.x, af.y, a.y);
}

// Pair (gx, gy) of the radius-2 region outside the tile, h < NPAIR_HALO:
// the four full halo rows as 18 pairs each, then the column pairs (0, 1)
// and (34, 35) of the tile rows.
__device__ __forceinline__ void halo_pair_coord(int h, int &gx, int &gy) {
    if (h < 72) {
        const int r = h / 18;
        gx = 2 * (h - 18 * r);
        gy = r < 2 ? r : PTY + r;
    } else {
        const int j = h - 72;
        gy = 2 + (j >> 1);
        gx = (j & 1) ? 34 : 0;
    }
}

// ---------------------------------------------------------------- stage X, pairs
// Where the pair's populations go: in-plane offsets of the rows y - 1, y,
// y + 1 and of the columns x - 1, x, x + 1 (first cell) and x, x + 1, x + 2
// (second cell), all wrapped; densities for the reduced storage forms.
struct PairPush {
    u32 row[3], col0[3], col1[3];
    int LxLy;
    u32 q_plane;             // q * Lx * Ly
    const float2 *ring[3];   // density ring slots of planes q-1, q, q+1 (tracked offsets)
    int idx;
    float2 ownA, ownB;       // the pair's densities
    bool track;
    float r0[2];
    unsigned seed;           // the instance's step count (stochastic rounding)
};

// Component s of population `dir` into cells c0 and c1 (at p0 and p1,
// adjacent when `adjacent`): vector stores rounding to nearest, or for
// BF16 one stochastically rounded store per cell with the random bits the
// one-cell kernel draws for that cell, direction and step.
template <typename T>
__device__ __forceinline__ void store_pair(T *p0, T *p1, float2 v, bool adjacent, u32 c0, u32 c1, int dir, int s,
                                           unsigned seed) {
    if (Store<T>::sround) {
        Store<T>::st_sr(p0, v.x, sround_bits(c0, dir, seed) >> (16 * s));
        Store<T>::st_sr(p1, v.y, sround_bits(c1, dir, seed) >> (16 * s));
    } else if (adjacent) {
        Pair<T>::stg(p0, v);
    } else {
        Store<T>::st(p0, v.x);
        Store<T>::st(p1, v.y);
    }
}

template <typename T>
__device__ __forceinline__ float2 pair_dest_offset(const PairPush &P, int s, int d, bool wall) {
    if (!P.track) return bc(P.r0[s]);
    if (wall) return s == 0 ? P.ownA : P.ownB;
    const float2 *rs = P.ring[cz(d) + 1] + P.idx + cx(d) + cy(d) * PG::RX;
    const float2 a = rs[0], b = rs[1];
    return s == 0 ? make_float2(a.x, b.x) : make_float2(a.y, b.y);
}

template <typename T, bool WALLS>
__device__ __forceinline__ void push2(T *__restrict__ fdst, u32 S, int s, int d, float2 v, float2 rs,
                                      const PairPush &P, bool bottom, bool top, float Uw) {
    if (WALLS && ((cz(d) < 0 && bottom) || (cz(d) > 0 && top))) {
        // halfway bounce-back into the cell itself, moving-wall term
        v = fma2(bc(-6.f * wq(d) * (float)cx(d) * (cz(d) < 0 ? -Uw : Uw)), rs, v);
        if (Store<T>::offset) v = fma2(bc(-wq(d)), pair_dest_offset<T>(P, s, d, true), v);
        const u32 dst = P.q_plane + P.row[1] + P.col0[1];
        T *p = fdst + (u32)((s * Q + opp(d)) * S + dst);
        store_pair<T>(p, p + 1, v, true, dst, dst + 1, opp(d), s, P.seed);
        return;
    }
    if (Store<T>::offset) v = fma2(bc(-wq(d)), pair_dest_offset<T>(P, s, d, false), v);
    const u32 plane = P.q_plane + (u32)(cz(d) * P.LxLy) + P.row[cy(d) + 1];
    T *base = fdst + (u32)((s * Q + d) * S);
    const u32 c0 = plane + P.col0[cx(d) + 1], c1 = plane + P.col1[cx(d) + 1];
    store_pair<T>(base + c0, base + c1, v, cx(d) == 0, c0, c1, d, s, P.seed);
}

// BGK + Guo collision of one component of the pair and push streaming (the
// pair-symmetric form of the one-cell kernel, on packed FP32).
template <typename T, bool WALLS>
__device__ __forceinline__ void collide_push2(const float2 *fv, T *__restrict__ fdst, u32 S, int s, float2 rs,
                                              const PairPush &P, const float2 u[3], const float2 F[3], float2 om,
                                              bool bottom, bool top, float Uw) {
    const float2 omc = sub2(bc(1.f), om), pref = fma2(bc(-0.5f), om, bc(1.f));
    const float2 uu = fma2(u[2], u[2], fma2(u[1], u[1], mul2(u[0], u[0])));
    const float2 uF = fma2(u[2], F[2], fma2(u[1], F[1], mul2(u[0], F[0])));
    const float2 E = fma2(bc(-3.f), mul2(pref, uF), mul2(om, mul2(rs, fma2(bc(-1.5f), uu, bc(1.f)))));
    const float2 orho = mul2(om, rs);
    {
        float2 v = fma2(omc, fv[0], mul2(bc(wq(0)), E));
        if (Store<T>::offset) {
            const float2 o = P.track ? (s == 0 ? P.ownA : P.ownB) : bc(P.r0[s]);
            v = fma2(bc(-wq(0)), o, v);
        }
        const u32 c0 = P.q_plane + P.row[1] + P.col0[1];
        T *p = fdst + (u32)(s * Q * S + c0);
        store_pair<T>(p, p + 1, v, true, c0, c0 + 1, 0, s, P.seed);
    }
    float2 Ew[2], a1w[2], b1w[2], a2w[2], b2w[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const float w = wq(c == 0 ? 1 : 7);
        Ew[c] = mul2(bc(w), E);
        a1w[c] = mul2(bc(4.5f * w), orho);
        b1w[c] = mul2(bc(9.f * w), pref);
        a2w[c] = mul2(bc(3.f * w), orho);
        b2w[c] = mul2(bc(3.f * w), pref);
    }
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const int c = i <= 6 ? 0 : 1;
        float2 cu = make_float2(0.f, 0.f), cF = cu;
        bool first = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int ca = a == 0 ? cx(i) : (a == 1 ? cy(i) : cz(i));
            if (!ca) continue;
            if (first) {
                cu = ca > 0 ? u[a] : mul2(bc(-1.f), u[a]);
                cF = ca > 0 ? F[a] : mul2(bc(-1.f), F[a]);
                first = false;
            } else {
                cu = ca > 0 ? add2(cu, u[a]) : sub2(cu, u[a]);
                cF = ca > 0 ? add2(cF, F[a]) : sub2(cF, F[a]);
            }
        }
        const float2 sym = fma2(cu, fma2(a1w[c], cu, mul2(b1w[c], cF)), Ew[c]);
        const float2 anti = fma2(a2w[c], cu, mul2(b2w[c], cF));
        push2<T, WALLS>(fdst, S, s, i, fma2(omc, fv[i], add2(sym, anti)), rs, P, bottom, top, Uw);
        push2<T, WALLS>(fdst, S, s, i + 1, fma2(omc, fv[i + 1], sub2(sym, anti)), rs, P, bottom, top, Uw);
    }
}

}  // namespace

template <typename T>
__global__ void __launch_bounds__(PNT, 1) k_fused_pair(const __grid_constant__ StepArgs A) {
    constexpr int TX = 32, RX = PG::RX, RY = PG::RY, R2N = PG::R2N;
    using Rg = Ring<PTY>;
    __shared__ u32 s_rows[RY];   // in-plane offsets of the radius-2 rows (wrapped)
    __shared__ u32 s_cols[RX];   // x of the radius-2 columns (wrapped)
    __shared__ u32 s_tmem;
    __shared__ __align__(8) unsigned long long s_bar;

    const int t = threadIdx.x, lx = t & 15, ty = t >> 4, warp = t >> 5;
    const int gx0 = 2 + 2 * lx, gy0 = 2 + ty;
    const int idx_in = gy0 * RX + gx0;   // ring index of the first cell (even)
    const int e_in = ty * 32 + 2 * lx;   // staging index of the first cell
    const u32 smem_base = smem_addr(lbfe_smem4);
    const u32 stage_addr = (smem_base + (u32)(sizeof(float) * PG::FLOATS) + 127u) & ~127u;
    const T *stage = reinterpret_cast<const T *>(reinterpret_cast<const char *>(lbfe_smem4) + (stage_addr - smem_base));
    const u32 bar = smem_addr(&s_bar);
    u32 parity = 0;                  // phase parity of the next copy to wait for
    u32 issued = 0;                  // copies issued (thread 0)
    bool expired = false;            // this thread's wait expired: no further waits or copies

    if (warp == 0) tm_alloc(&s_tmem, P_TMEM_COLS);
    if (t == 0) mbar_init(bar);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    // this warp's TMEM columns: lane quarter warp % 4, 256 columns from (warp / 4) * 256
    const u32 tm_warp = s_tmem + ((u32)(32 * (warp & 3)) << 16) + (u32)((warp >> 2) * 256);

    __shared__ int s_item[2];   // work items from the launch's counter, one ahead
    if (t == 0) {
        const int first = blockIdx.x;
        s_item[0] = first;
        if (first < A.total_items) {
            const ItemPos P0 = item_pos<PTY>(A, first);
            if (A.inst[P0.k].tma) {
                issue_plane<T, PTY>(A, P0, P0.z0 - 2, stage_addr, bar);
                ++issued;
            }
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
        const ItemPos P = item_pos<PTY>(A, item);
        const StepInst &I = A.inst[P.k];
        const int Lx = I.Lx, Ly = I.Ly, Lz = I.Lz;
        const int LxLy = I.LxLy;
        const u32 S = I.S;
        const int bx = P.bx, by = P.by, z0 = P.z0, z1 = P.z1;
        const int x0 = bx * TX - 2, y0 = by * PTY - 2;
        const bool tma = I.tma != 0;
        const T *__restrict__ fin = (const T *)I.fin;
        T *__restrict__ fout = (T *)I.fout;
        const float *__restrict__ Cin = I.Cin;
        float *__restrict__ Cout = I.Cout;
        const float Uw = I.Uw;

        __syncthreads();
        if (t < RY) s_rows[t] = (u32)(wrapg(y0 + t, Ly) * Lx);
        if (t < RX) s_cols[t] = (u32)wrapg(x0 + t, Lx);
        __syncthreads();

        const int x = bx * TX + 2 * lx, y = by * PTY + ty;
        const bool valid = x < Lx && y < Ly;   // Lx even: the second cell is valid with the first
        PairPush Pp;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Pp.row[a] = s_rows[gy0 - 1 + a];
            Pp.col0[a] = s_cols[gx0 - 1 + a];
            Pp.col1[a] = s_cols[gx0 + a];
        }
        const u32 ofs_in = Pp.row[1] + Pp.col0[1];
        Pp.LxLy = LxLy;
        Pp.idx = idx_in;
        Pp.track = I.dens_out != nullptr;
        // the instance's step count: the seed of the BF16 stochastic rounding
        Pp.seed = step_seed<Store<T>::sround>(A, I, P.k, item, t);
        Pp.r0[0] = I.rho0A;
        Pp.r0[1] = I.rho0B;
        // this thread's halo pair
        const bool has_halo = t < NPAIR_HALO;
        u32 h_ofs = 0;
        int h_idx = 0;
        {
            int gx, gy;
            halo_pair_coord(has_halo ? t : 0, gx, gy);
            h_ofs = s_rows[gy] + s_cols[gx];
            h_idx = gy * RX + gx;
        }

        float2 FA[3], FB[3], uo[3], rAo = bc(1.f), rBo = bc(0.f);

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

            // ---------------- stage M(p)
            {
                const u32 pl = (u32)(min(max(p, 0), Lz - 1) * LxLy);
                if (has_halo) {
                    MPair m;
                    m_load2<T>(I, fin, Cin, S, pl + h_ofs, m);
                    m_store2(I, m, h_idx, L.r3[2], ring2(p), L.cf[2]);
                }
                if (tma) {
                    if (!expired && !mbar_wait(bar, parity)) expired = true;
                    parity ^= 1u;
                }
                {
                    MPair m;
                    if (tma && valid)
                        m_load2_staged<T>(I, stage, e_in, Cin, S, pl + ofs_in, m);
                    else
                        m_load2<T>(I, fin, Cin, S, pl + ofs_in, m);
                    m_store2(I, m, idx_in, L.r3[2], ring2(p), L.cf[2]);
                    tm_store76(tm_warp + (u32)((p & 1) * 128), m.f);
                }
            }
            __syncthreads();
            if (t == 0) {
                if (p == z0 - 2) s_item[slot ^ 1] = next_t0;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                if (p < z1 + 1) {
                    if (tma) {
                        issue_plane<T, PTY>(A, P, p + 1, stage_addr, bar, expired ? 0u : 1u);
                        issued += expired ? 0u : 1u;
                    }
                } else if (next_t0 < A.total_items) {
                    const ItemPos Pn = item_pos<PTY>(A, next_t0);
                    if (A.inst[Pn.k].tma) {
                        issue_plane<T, PTY>(A, Pn, Pn.z0 - 2, stage_addr, bar, expired ? 0u : 1u);
                        issued += expired ? 0u : 1u;
                    }
                }
            }
            // ---------------- stage F(q): the pair, then the radius-1 ring
            if (q >= max(z0 - 1, 0) && q <= min(z1, Lz - 1)) {
                float a0[3], b0[3], u0[3], a1[3], b1[3], u1[3], ra0, rb0, ra1, rb1;
                stage_f_cell<PTY>(I, idx_in, L, a0, b0, u0, ra0, rb0);
                stage_f_cell<PTY>(I, idx_in + 1, L, a1, b1, u1, ra1, rb1);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    FA[a] = make_float2(a0[a], a1[a]);
                    FB[a] = make_float2(b0[a], b1[a]);
                    uo[a] = make_float2(u0[a], u1[a]);
                }
                rAo = make_float2(ra0, ra1);
                rBo = make_float2(rb0, rb1);
                for (int h = t; h < PG::NRING1; h += PNT) {
                    int gx, gy;
                    ring1_coord<PTY>(h, gx, gy);
                    float a[3], b[3], uu[3], ra, rb;
                    stage_f_cell<PTY>(I, gy * RX + gx, L, a, b, uu, ra, rb);
                }
            }
            // ---------------- stage X(q)
            if (q >= z0 && q < z1) {
                float2 fx[2 * Q];
                tm_load76(tm_warp + (u32)((q & 1) * 128), fx);   // whole warp
                if (valid) {
                    const float2 rt = add2(rAo, rBo);
                    bool bad = !(rt.x > 0.f) || !(rt.y > 0.f);
#pragma unroll
                    for (int a = 0; a < 3; ++a) bad |= (uo[a].x != uo[a].x) || (uo[a].y != uo[a].y);
                    if (bad) raise_step_flag(A.status, I, kFlagDiverged);
                    float2 om;
                    om.x = 1.0f / (3.0f * ((rAo.x * I.nu_A + rBo.x * I.nu_B) / rt.x) + 0.5f);
                    om.y = 1.0f / (3.0f * ((rAo.y * I.nu_A + rBo.y * I.nu_B) / rt.y) + 0.5f);
                    const bool bottom = q == 0, top = q == Lz - 1;
                    Pp.q_plane = (u32)(q * LxLy);
                    const float2 *rho_s = reinterpret_cast<const float2 *>(smem() + Rg::RHO);
                    Pp.ring[0] = rho_s + L.r3[0] * R2N;
                    Pp.ring[1] = rho_s + L.r3[1] * R2N;
                    Pp.ring[2] = rho_s + L.r3[2] * R2N;
                    Pp.ownA = rAo;
                    Pp.ownB = rBo;
                    if (bottom || top) {
                        collide_push2<T, true>(fx, fout, S, 0, rAo, Pp, uo, FA, om, bottom, top, Uw);
                        collide_push2<T, true>(fx + Q, fout, S, 1, rBo, Pp, uo, FB, om, bottom, top, Uw);
                    } else {
                        collide_push2<T, false>(fx, fout, S, 0, rAo, Pp, uo, FA, om, false, false, Uw);
                        collide_push2<T, false>(fx + Q, fout, S, 1, rBo, Pp, uo, FB, om, false, false, Uw);
                    }
                    if (Store<T>::offset && Pp.track)
                        *reinterpret_cast<float4 *>(I.dens_out + Pp.q_plane + ofs_in) =
                            make_float4(rAo.x, rBo.x, rAo.y, rBo.y);
                }
            }
            // ---------------- stage U(r): no barrier before it (u of plane q
            // is read at the thread's own cells only)
            if (r >= z0 && r < z1 && valid) {
                float c0[6], c1[6];
                bool ok = stage_u_cell<PTY>(I, idx_in, L, r, c0);
                ok &= stage_u_cell<PTY>(I, idx_in + 1, L, r, c1);
                if (!ok) raise_step_flag(A.status, I, kFlagDiverged);
                const u32 n = (u32)(r * LxLy) + ofs_in;
#pragma unroll
                for (int q6 = 0; q6 < 6; ++q6)
                    *reinterpret_cast<float2 *>(Cout + (u32)(q6 * S + n)) = make_float2(c0[q6], c1[q6]);
            }
            __syncthreads();
        }
        item = s_item[slot ^ 1];   // published in the first iteration, several barriers ago
        slot ^= 1;
    }

    if (t == 0 && A.total_items > (int)gridDim.x) release_work_counters(A.work);
    if (expired) {
        // thread 0: the copy whose wait expired may still be in flight: wait
        // for its phase once more, bounded, before the shared memory is
        // released
        if (t == 0 && issued > 0) mbar_wait(bar, (issued - 1u) & 1u);
        atomicOr(A.status, kFlagTimeout);
    }
    tm_wait_st();   // no TMEM store may be pending when the columns are freed
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    if (warp == 0) tm_dealloc(s_tmem, P_TMEM_COLS);
}

namespace {

template <typename T>
constexpr size_t pair_smem_bytes() {
    return sizeof(float) * PG::FLOATS + 128 + sizeof(T) * 2 * Q * 512;
}

template <typename T>
cudaError_t pair_prep_t(int *bps) {
    const size_t smem = pair_smem_bytes<T>();
    cudaError_t e = cudaFuncSetAttribute(k_fused_pair<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int b = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_fused_pair<T>, PNT, smem);
    if (e != cudaSuccess) return e;
    *bps = b < 1 ? b : 1;   // all 512 TMEM columns per block
    return cudaSuccess;
}

}  // namespace

cudaError_t step_pair_launch(const StepArgs &a, int grid, int precision, cudaStream_t st) {
    switch (precision) {
        case LBFE_FP16_OFFSET:
            k_fused_pair<__half><<<grid, PNT, pair_smem_bytes<__half>(), st>>>(a);
            break;
        case LBFE_BF16_OFFSET:
            k_fused_pair<__nv_bfloat16><<<grid, PNT, pair_smem_bytes<__nv_bfloat16>(), st>>>(a);
            break;
        default:
            k_fused_pair<float><<<grid, PNT, pair_smem_bytes<float>(), st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t step_pair_prepare(int precision, int *blocks_per_sm) {
    switch (precision) {
        case LBFE_FP16_OFFSET: return pair_prep_t<__half>(blocks_per_sm);
        case LBFE_BF16_OFFSET: return pair_prep_t<__nv_bfloat16>(blocks_per_sm);
        default: return pair_prep_t<float>(blocks_per_sm);
    }
}

}  // namespace lbfe
