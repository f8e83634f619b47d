// kernels.cuh -- hand-written sm_103a kernels of the nested block solver:
// block-sparse products with fused epilogues, deterministic multi-dot /
// multi-axpy for CGS2 Arnoldi, the device Givens least-squares update and the
// AMG transfer operators.  Internal header (templates), included by the
// translation units that launch them.
#pragma once

#include <cstring>
#include <type_traits>

#include "nbp_common.cuh"

namespace nbp {

// ===================================================== block-sparse products
// y = epilogue(M x) for a block CSR matrix with BR x BC blocks.  A group of G
// lanes walks one block row's values as one flat, contiguous array (perfectly
// coalesced loads whatever the block shape), keeps BR partial sums, and
// reduces them with xor shuffles inside the group.  Epilogues:
//   EPI_SET  y = Mx (+ rank-one term, LR)      EPI_ADD  y += Mx
//   EPI_SUB  y -= Mx                           EPI_RES  y = b - Mx
//   EPI_CHEB r = b - Mx; d = c1 d + c2 Dinv r; xout = x + d   (Chebyshev step)
enum Epi { EPI_SET = 0, EPI_ADD = 1, EPI_SUB = 2, EPI_RES = 3, EPI_CHEB = 4 };

struct SpmvArgs {
    int nbr;
    const int *rp, *ci;
    const void *val;
    const void *x;
    void *y;
    const void *b;          // EPI_RES / EPI_CHEB
    const void *dinv;       // EPI_CHEB: BR x BR per row (same type as vectors)
    void *d;                // EPI_CHEB: Chebyshev direction (in/out)
    void *xout;             // EPI_CHEB: x + d
    double c1, c2;          // EPI_CHEB coefficients (FP64 vectors)
    float c1f, c2f;         // the same, pre-rounded for FP32 vectors (no FP64 work per element)
    const int *lr_rp, *lr_k, *lr_c;   // rank-one epilogue (EPI_SET only)
    const double *lr_val, *lr_f;
    int nslice;                       // sliced-ELL layout (k_sell): slices of C rows
    const long long *sl_ptr;
    const int *sl_ci;
};

template <int BR, int BC, int G, typename VT, typename XT, int EPI, bool LR>
__global__ void __launch_bounds__(256) k_bspmv(SpmvArgs a) {
    using AT = XT;   // accumulate in the vector type (FP64 or FP32)
    constexpr int BB = BR * BC;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int row = (int)(gid / G);
    const int lane = (int)(gid % G);
    if (row >= a.nbr) return;   // whole groups leave together (G divides 32)
    const unsigned wl = threadIdx.x & 31u;
    const unsigned mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (wl & ~(unsigned)(G - 1)));
    const int e0 = __ldg(a.rp + row);
    const int cnt = (__ldg(a.rp + row + 1) - e0) * BB;
    const VT *__restrict__ val = (const VT *)a.val + (long long)e0 * BB;
    const int *__restrict__ ci = a.ci + e0;
    const XT *__restrict__ x = (const XT *)a.x;
    AT acc0 = 0, acc1 = 0, acc2 = 0;
#pragma unroll 4
    for (int v = lane; v < cnt; v += G) {
        const int e = v / BB;
        const int rc = v - e * BB;
        const int r = rc / BC;
        const int c = rc - r * BC;
        const AT p = cvt<AT>(__ldg(val + v)) * __ldg(x + (long long)__ldg(ci + e) * BC + c);
        if (BR == 1) acc0 += p;
        else {
            acc0 += (r == 0) ? p : AT(0);
            acc1 += (r == 1) ? p : AT(0);
            acc2 += (r == 2) ? p : AT(0);
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        acc0 += __shfl_xor_sync(mask, acc0, o);
        if (BR > 1) {
            acc1 += __shfl_xor_sync(mask, acc1, o);
            acc2 += __shfl_xor_sync(mask, acc2, o);
        }
    }
    if (lane >= BR) return;
    AT s = (lane == 0) ? acc0 : (lane == 1 ? acc1 : acc2);
    const long long idx = (long long)row * BR + lane;
    XT *y = (XT *)a.y;
    if (EPI == EPI_SET) {
        if (LR) {   // FP64 only on the rows that carry rank-one entries
            const int e0 = a.lr_rp[row], e1 = a.lr_rp[row + 1];
            if (e1 > e0) {
                double t = 0.0;
                for (int q = e0; q < e1; ++q)
                    if (a.lr_c[q] == lane) t += a.lr_f[a.lr_k[q]] * a.lr_val[q];
                s = (AT)((double)s + t);
            }
        }
        y[idx] = s;
    } else if (EPI == EPI_ADD) {
        y[idx] += s;
    } else if (EPI == EPI_SUB) {
        y[idx] -= s;
    } else if (EPI == EPI_RES) {
        y[idx] = ((const XT *)a.b)[idx] - s;
    } else {   // EPI_CHEB, BR == BC
        const XT *b = (const XT *)a.b;
        const XT *dinv = (const XT *)a.dinv + (long long)row * BR * BR + lane * BR;
        AT t;
        if (BR == 1) {
            t = dinv[0] * (b[idx] - s);
        } else {
            const AT r0 = b[(long long)row * 3 + 0] - acc0;
            const AT r1 = b[(long long)row * 3 + 1] - acc1;
            const AT r2 = b[(long long)row * 3 + 2] - acc2;
            t = dinv[0] * r0 + dinv[1] * r1 + dinv[2] * r2;
        }
        XT *d = (XT *)a.d;
        const AT c1 = sizeof(AT) == 4 ? (AT)a.c1f : (AT)a.c1, c2 = sizeof(AT) == 4 ? (AT)a.c2f : (AT)a.c2;
        const AT dn = c1 * d[idx] + c2 * t;
        d[idx] = dn;
        ((XT *)a.xout)[idx] = x[idx] + dn;
    }
}

// Streamed loads of matrix values and columns: each is read once per
// product, so they can bypass L1 allocation (ld.global.nc.L1::no_allocate)
// and leave L1 to the x gathers, which neighbouring rows share.
__device__ __forceinline__ float lds(const float *p) {
    float v;
    asm volatile("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ double lds(const double *p) {
    double v;
    asm volatile("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ int lds(const int *p) {
    int v;
    asm volatile("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ int2 lds(const int2 *p) {
    int2 v;
    asm volatile("ld.global.nc.L1::no_allocate.v2.s32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ __nv_bfloat16 lds(const __nv_bfloat16 *p) {
    unsigned short v;
    asm volatile("ld.global.nc.L1::no_allocate.b16 %0, [%1];" : "=h"(v) : "l"(p));
    __nv_bfloat16 r;
    memcpy(&r, &v, 2);
    return r;
}
__device__ __forceinline__ __nv_bfloat162 lds(const __nv_bfloat162 *p) {
    unsigned v;
    asm volatile("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(p));
    __nv_bfloat162 r;
    memcpy(&r, &v, 4);
    return r;
}

// Matrix loads of the sliced layouts: streamed (no L1 allocation) for
// 32-row slices, whose warps read whole 128-byte segments; 8-row slices read
// quarter segments, and there the lines that L1 keeps serve the neighbouring
// components, so those loads stay cached.
template <bool STREAM, typename P> __device__ __forceinline__ P ldm(const P *p) {
    if constexpr (STREAM) return lds(p);
    else return __ldg(p);
}

// One pair of slots of the paired BF16 layout: columns c, values m, added in
// slot order (the first slot of the pair, then the second).
template <int BS>
__device__ __forceinline__ void pair_fma(const int2 c, const __nv_bfloat162 (&m)[BS * BS], const float *__restrict__ x,
                                         float &acc0, float &acc1, float &acc2) {
    if (BS == 1) {
        const float2 mm = __bfloat1622float2(m[0]);
        acc0 += mm.x * __ldg(x + c.x);
        acc0 += mm.y * __ldg(x + c.y);
    } else {
        const float xa0 = __ldg(x + 3LL * c.x), xa1 = __ldg(x + 3LL * c.x + 1), xa2 = __ldg(x + 3LL * c.x + 2);
        const float xb0 = __ldg(x + 3LL * c.y), xb1 = __ldg(x + 3LL * c.y + 1), xb2 = __ldg(x + 3LL * c.y + 2);
        float2 mm[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) mm[q] = __bfloat1622float2(m[q]);
        acc0 += mm[0].x * xa0 + mm[1].x * xa1 + mm[2].x * xa2;
        acc1 += mm[3].x * xa0 + mm[4].x * xa1 + mm[5].x * xa2;
        acc2 += mm[6].x * xa0 + mm[7].x * xa1 + mm[8].x * xa2;
        acc0 += mm[0].y * xb0 + mm[1].y * xb1 + mm[2].y * xb2;
        acc1 += mm[3].y * xb0 + mm[4].y * xb1 + mm[5].y * xb2;
        acc2 += mm[6].y * xb0 + mm[7].y * xb1 + mm[8].y * xb2;
    }
}

// Slots p0, p0 + step, ... of the paired BF16 layout (DMat::sl2_ptr) of one
// row: per pair, one int2 of columns and one bf16x2 per component; the two
// slots are added in slot order, as the unpaired loop adds them.  Two pairs
// are loaded before either is used (more loads in flight per thread); the
// pairs are still added in ascending order.
template <int BS, int C>
__device__ __forceinline__ void sell_pairs(const SpmvArgs &a, long long base2, int np, int t, int p0, int step,
                                           const float *__restrict__ x, float &acc0, float &acc1, float &acc2) {
    constexpr int BB = BS * BS;
    const __nv_bfloat162 *__restrict__ val = (const __nv_bfloat162 *)a.val;
    const int2 *__restrict__ ci = (const int2 *)a.sl_ci;
    int p = p0;
    // 32-row slices (the fine level, HBM-bound): two pairs per step; 8-row
    // slices (coarse levels) measured faster one pair at a time
    if (C == 32) {
        for (; p + step < np; p += 2 * step) {
            const long long g0 = base2 + (long long)C * p, g1 = g0 + (long long)C * step;
            const int2 c0 = ldm<C == 32>(ci + g0 + t), c1 = ldm<C == 32>(ci + g1 + t);
            __nv_bfloat162 m0[BB], m1[BB];
#pragma unroll
            for (int q = 0; q < BB; ++q) m0[q] = ldm<C == 32>(val + g0 * BB + t + q * C);
#pragma unroll
            for (int q = 0; q < BB; ++q) m1[q] = ldm<C == 32>(val + g1 * BB + t + q * C);
            pair_fma<BS>(c0, m0, x, acc0, acc1, acc2);
            pair_fma<BS>(c1, m1, x, acc0, acc1, acc2);
        }
    }
    for (; p < np; p += step) {
        const long long g0 = base2 + (long long)C * p;
        const int2 c0 = ldm<C == 32>(ci + g0 + t);
        __nv_bfloat162 m0[BB];
#pragma unroll
        for (int q = 0; q < BB; ++q) m0[q] = ldm<C == 32>(val + g0 * BB + t + q * C);
        pair_fma<BS>(c0, m0, x, acc0, acc1, acc2);
    }
}

// The unpaired last slot of an odd-width slice of the paired layout: its
// columns at sl_ci[g + t] and value q at val[g bb + C q + t] (int and bf16
// units), g = the slice's slot offset + C (width - 1).
template <int BS, int C>
__device__ __forceinline__ void sell_single(const SpmvArgs &a, long long g, int t, const float *__restrict__ x,
                                            float &acc0, float &acc1, float &acc2) {
    const __nv_bfloat16 *__restrict__ val = (const __nv_bfloat16 *)a.val + g * (BS * BS) + t;
    const int c = ldm<C == 32>(a.sl_ci + g + t);
    if (BS == 1) {
        acc0 += __bfloat162float(ldm<C == 32>(val)) * __ldg(x + c);
    } else {
        const float x0 = __ldg(x + 3LL * c), x1 = __ldg(x + 3LL * c + 1), x2 = __ldg(x + 3LL * c + 2);
        float m[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) m[q] = __bfloat162float(ldm<C == 32>(val + q * C));
        acc0 += m[0] * x0 + m[1] * x1 + m[2] * x2;
        acc1 += m[3] * x0 + m[4] * x1 + m[5] * x2;
        acc2 += m[6] * x0 + m[7] * x1 + m[8] * x2;
    }
}

// Sliced-ELL product for square BS x BS blocks: one thread per block row, C
// rows per slice (C = 32: a warp per slice; C = 8 for matrices whose row
// lengths vary, to cut padding).  Every load of values and columns by the C
// threads of a slice is one contiguous segment (C x value bytes).  Same
// epilogues as k_bspmv (a.rp unused; a.sl_* describe the slices).
template <int BS, typename VT, typename XT, int EPI, bool LR, int C>
__global__ void __launch_bounds__(256) k_sell(SpmvArgs a) {
    using AT = XT;
    constexpr int BB = BS * BS;
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int sl = row / C, t = row % C;
    if (sl >= a.nslice) return;
    const long long base = a.sl_ptr[sl];
    const int w = (int)((a.sl_ptr[sl + 1] - base) / C);
    const VT *__restrict__ val = (const VT *)a.val;
    const int *__restrict__ ci = a.sl_ci;
    const XT *__restrict__ x = (const XT *)a.x;
    AT acc0 = 0, acc1 = 0, acc2 = 0;
    if constexpr (std::is_same<VT, __nv_bfloat16>::value) {   // paired layout: w / 2 pairs, then one slot if w is odd
        sell_pairs<BS, C>(a, base / 2, w / 2, t, 0, 1, x, acc0, acc1, acc2);
        if (w & 1) sell_single<BS, C>(a, base + (long long)C * (w - 1), t, x, acc0, acc1, acc2);
    } else {
#pragma unroll 2
        for (int k = 0; k < w; ++k) {
            const long long g = base + (long long)C * k;
            const int c = ldm<C == 32>(ci + g + t);
            const VT *v = val + g * BB + t;
            if (BS == 1) {
                acc0 += cvt<AT>(ldm<C == 32>(v)) * __ldg(x + c);
            } else {
                const AT x0 = __ldg(x + 3LL * c), x1 = __ldg(x + 3LL * c + 1), x2 = __ldg(x + 3LL * c + 2);
                acc0 += cvt<AT>(ldm<C == 32>(v)) * x0 + cvt<AT>(ldm<C == 32>(v + C)) * x1 + cvt<AT>(ldm<C == 32>(v + 2 * C)) * x2;
                acc1 += cvt<AT>(ldm<C == 32>(v + 3 * C)) * x0 + cvt<AT>(ldm<C == 32>(v + 4 * C)) * x1 + cvt<AT>(ldm<C == 32>(v + 5 * C)) * x2;
                acc2 += cvt<AT>(ldm<C == 32>(v + 6 * C)) * x0 + cvt<AT>(ldm<C == 32>(v + 7 * C)) * x1 + cvt<AT>(ldm<C == 32>(v + 8 * C)) * x2;
            }
        }
    }
    if (row >= a.nbr) return;
    AT accs[3] = {acc0, acc1, acc2};
    XT *y = (XT *)a.y;
    const bool lr = LR && EPI == EPI_SET;
    const int lr0 = lr ? a.lr_rp[row] : 0, lr1 = lr ? a.lr_rp[row + 1] : 0;
    if (EPI == EPI_CHEB) {
        const XT *b = (const XT *)a.b;
        const XT *dinv = (const XT *)a.dinv + (long long)row * BB;
        XT *d = (XT *)a.d;
        XT *xo = (XT *)a.xout;
        const AT c1 = sizeof(AT) == 4 ? (AT)a.c1f : (AT)a.c1, c2 = sizeof(AT) == 4 ? (AT)a.c2f : (AT)a.c2;
        AT r[3];
#pragma unroll
        for (int q = 0; q < BS; ++q) r[q] = b[(long long)row * BS + q] - accs[q];
#pragma unroll
        for (int q = 0; q < BS; ++q) {
            AT tq = 0;
#pragma unroll
            for (int c = 0; c < BS; ++c) tq += dinv[q * BS + c] * r[c];
            const long long idx = (long long)row * BS + q;
            const AT dn = c1 * d[idx] + c2 * tq;
            d[idx] = dn;
            xo[idx] = x[idx] + dn;
        }
        return;
    }
#pragma unroll
    for (int q = 0; q < BS; ++q) {
        const long long idx = (long long)row * BS + q;
        AT s = accs[q];
        if (EPI == EPI_SET) {
            // the rank-one term in FP64, only on the rows that carry its
            // entries (outlet rows): GB300's FP64 pipe would otherwise hold
            // every warp for the conversions of every row
            if (lr && lr1 > lr0) {
                double tt = 0.0;
                for (int e = lr0; e < lr1; ++e)
                    if (a.lr_c[e] == q) tt += a.lr_f[a.lr_k[e]] * a.lr_val[e];
                s = (AT)((double)s + tt);
            }
            y[idx] = s;
        } else if (EPI == EPI_ADD) {
            y[idx] += s;
        } else if (EPI == EPI_SUB) {
            y[idx] -= s;
        } else {
            y[idx] = ((const XT *)a.b)[idx] - s;
        }
    }
}

// Sliced-ELL product for the rectangular coupling blocks (B: 3x1, C: 1x3):
// one thread per block row, slot values component-major as in k_sell (value
// q = r BC + c of the C slots at (slot base) * BR BC + C q + t).  Epilogues
// SET / ADD / SUB; FP64 or FP32 values.
template <int BR, int BC, typename VT, typename XT, int EPI, int C>
__global__ void __launch_bounds__(256) k_sellr(SpmvArgs a) {
    using AT = XT;
    constexpr int BB = BR * BC;
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int sl = row / C, t = row % C;
    if (sl >= a.nslice) return;
    const long long base = a.sl_ptr[sl];
    const int w = (int)((a.sl_ptr[sl + 1] - base) / C);
    const VT *__restrict__ val = (const VT *)a.val;
    const int *__restrict__ ci = a.sl_ci;
    const XT *__restrict__ x = (const XT *)a.x;
    AT acc[BR];
#pragma unroll
    for (int r = 0; r < BR; ++r) acc[r] = 0;
#pragma unroll 2
    for (int k = 0; k < w; ++k) {
        const long long g = base + (long long)C * k;
        const int c = ldm<C == 32>(ci + g + t);
        const VT *v = val + g * BB + t;
        AT xs[BC];
#pragma unroll
        for (int cc = 0; cc < BC; ++cc) xs[cc] = __ldg(x + (long long)BC * c + cc);
#pragma unroll
        for (int r = 0; r < BR; ++r) {
            AT u = 0;
#pragma unroll
            for (int cc = 0; cc < BC; ++cc) u += cvt<AT>(ldm<C == 32>(v + (r * BC + cc) * C)) * xs[cc];
            acc[r] += u;
        }
    }
    if (row >= a.nbr) return;
    XT *y = (XT *)a.y;
#pragma unroll
    for (int r = 0; r < BR; ++r) {
        const long long idx = (long long)row * BR + r;
        if (EPI == EPI_SET) y[idx] = acc[r];
        else if (EPI == EPI_ADD) y[idx] += acc[r];
        else y[idx] -= acc[r];
    }
}

// Sliced-ELL product with T threads per block row (T = 2, 4, 8: thread h
// takes slots h, h + T, ..., then an xor-shuffle tree over the T lanes), for
// coarse levels whose rows are few, so that one thread per row leaves the
// SMs with little memory parallelism.  No rank-one epilogue (coarse levels
// need none).
constexpr int kSellMT = 1000;   // DMat::tuned code kSellMT + T selects this kernel with T threads per row
__host__ __device__ inline bool is_sellm(int g) { return g == kSellMT + 2 || g == kSellMT + 4 || g == kSellMT + 8; }
template <int BS, typename VT, typename XT, int EPI, int C, int T>
__global__ void __launch_bounds__(256) k_sellm(SpmvArgs a) {
    using AT = XT;
    constexpr int BB = BS * BS;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int row = (int)(gid / T), h = (int)(gid % T);
    const int sl = row / C, t = row % C;
    const bool live = sl < a.nslice;
    // the row's own epilogue operands are loaded before the slot loop, so that
    // their latency overlaps the gather chain (these small levels are
    // latency-bound: fewer rows than the GPU has threads in flight)
    const bool own = h == 0 && live && row < a.nbr;
    AT eb[3] = {0, 0, 0}, ed[3] = {0, 0, 0}, ex[3] = {0, 0, 0}, edi[BB];
    if (own && (EPI == EPI_RES || EPI == EPI_CHEB)) {
#pragma unroll
        for (int q = 0; q < BS; ++q) eb[q] = ((const XT *)a.b)[(long long)row * BS + q];
    }
    if (own && EPI == EPI_CHEB) {
        const XT *dv = (const XT *)a.dinv + (long long)row * BB;
#pragma unroll
        for (int q = 0; q < BS; ++q) {
            ed[q] = ((const XT *)a.d)[(long long)row * BS + q];
            ex[q] = ((const XT *)a.x)[(long long)row * BS + q];
        }
#pragma unroll
        for (int q = 0; q < BB; ++q) edi[q] = dv[q];
    }
    const long long base = live ? a.sl_ptr[sl] : 0;
    const int w = live ? (int)((a.sl_ptr[sl + 1] - base) / C) : 0;
    const VT *__restrict__ val = (const VT *)a.val;
    const int *__restrict__ ci = a.sl_ci;
    const XT *__restrict__ x = (const XT *)a.x;
    AT acc0 = 0, acc1 = 0, acc2 = 0;
    if constexpr (std::is_same<VT, __nv_bfloat16>::value) {   // paired layout: the T threads take alternate pairs
        sell_pairs<BS, C>(a, base / 2, w / 2, t, h, T, x, acc0, acc1, acc2);
        // an odd width's last slot goes to the thread whose turn comes next
        if ((w & 1) && h == (w / 2) % T) sell_single<BS, C>(a, base + (long long)C * (w - 1), t, x, acc0, acc1, acc2);
    } else {
        for (int k = h; k < w; k += T) {
            const long long g = base + (long long)C * k;
            const int c = ldm<C == 32>(ci + g + t);
            const VT *v = val + g * BB + t;
            if (BS == 1) {
                acc0 += cvt<AT>(ldm<C == 32>(v)) * __ldg(x + c);
            } else {
                const AT x0 = __ldg(x + 3LL * c), x1 = __ldg(x + 3LL * c + 1), x2 = __ldg(x + 3LL * c + 2);
                acc0 += cvt<AT>(ldm<C == 32>(v)) * x0 + cvt<AT>(ldm<C == 32>(v + C)) * x1 + cvt<AT>(ldm<C == 32>(v + 2 * C)) * x2;
                acc1 += cvt<AT>(ldm<C == 32>(v + 3 * C)) * x0 + cvt<AT>(ldm<C == 32>(v + 4 * C)) * x1 + cvt<AT>(ldm<C == 32>(v + 5 * C)) * x2;
                acc2 += cvt<AT>(ldm<C == 32>(v + 6 * C)) * x0 + cvt<AT>(ldm<C == 32>(v + 7 * C)) * x1 + cvt<AT>(ldm<C == 32>(v + 8 * C)) * x2;
            }
        }
    }
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) {
        acc0 += __shfl_xor_sync(0xffffffffu, acc0, o);
        if (BS > 1) {
            acc1 += __shfl_xor_sync(0xffffffffu, acc1, o);
            acc2 += __shfl_xor_sync(0xffffffffu, acc2, o);
        }
    }
    if (!own) return;
    const AT accs[3] = {acc0, acc1, acc2};
    XT *y = (XT *)a.y;
    if (EPI == EPI_CHEB) {
        XT *d = (XT *)a.d;
        XT *xo = (XT *)a.xout;
        const AT c1 = sizeof(AT) == 4 ? (AT)a.c1f : (AT)a.c1, c2 = sizeof(AT) == 4 ? (AT)a.c2f : (AT)a.c2;
        AT r[3];
#pragma unroll
        for (int q = 0; q < BS; ++q) r[q] = eb[q] - accs[q];
#pragma unroll
        for (int q = 0; q < BS; ++q) {
            AT tq = 0;
#pragma unroll
            for (int c = 0; c < BS; ++c) tq += edi[q * BS + c] * r[c];
            const long long idx = (long long)row * BS + q;
            const AT dn = c1 * ed[q] + c2 * tq;
            d[idx] = dn;
            xo[idx] = ex[q] + dn;
        }
        return;
    }
#pragma unroll
    for (int q = 0; q < BS; ++q) {
        const long long idx = (long long)row * BS + q;
        if (EPI == EPI_SET) y[idx] = accs[q];
        else if (EPI == EPI_ADD) y[idx] += accs[q];
        else if (EPI == EPI_SUB) y[idx] -= accs[q];
        else y[idx] = eb[q] - accs[q];
    }
}

// ============================================ deterministic reductions
// The Arnoldi kernels run on a fixed grid of kReduceBlocks blocks; block b
// covers one fixed contiguous chunk of the vectors (a multiple of the 16-byte
// vector width), writes its partial sums to partial[col][b], and the last
// block to finish (atomic ticket) adds the partials of every column in a
// fixed order.  Results therefore do not depend on block scheduling.

// 16-byte vectors of T (float4 / double2)
template <typename T> struct Vec16;
template <> struct Vec16<float> { static constexpr int W = 4; using type = float4; };
template <> struct Vec16<double> { static constexpr int W = 2; using type = double2; };

template <typename T> __device__ __forceinline__ void vld(const T *p, T (&o)[Vec16<T>::W]) {
    const typename Vec16<T>::type u = *reinterpret_cast<const typename Vec16<T>::type *>(p);
    memcpy(o, &u, 16);
}
template <typename T> __device__ __forceinline__ void vst(T *p, const T (&o)[Vec16<T>::W]) {
    typename Vec16<T>::type u;
    memcpy(&u, o, 16);
    *reinterpret_cast<typename Vec16<T>::type *>(p) = u;
}

// This block's chunk [lo, hi) of 0..n-1; lo is a multiple of W.
__device__ __forceinline__ void block_chunk(long long n, int W, long long &lo, long long &hi) {
    const long long per = ((n + gridDim.x - 1) / gridDim.x + W - 1) / W * W;
    lo = min(n, (long long)blockIdx.x * per);
    hi = min(n, lo + per);
}

// True in the last block of the grid to get here (after every block has
// published its partials).  The last block resets the ticket before it ends.
__device__ __forceinline__ bool grid_last_block(unsigned *ticket) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    return s_last != 0;
}

// out[col] = sum_b partial[col][b] for col < ncols, run by one whole block:
// thread t adds partials b = t, t + blockDim, ... of up to 8 columns at a time
// (all loads independent), then a warp tree and a fixed sum over the warps --
// one order whatever the scheduling.
// The FP32 kernels' partials are float-float pairs (float2 in the double
// slots); those go through block_reduce_partials_ff.
__device__ __forceinline__ void block_reduce_partials(const double *partial, int nb, int ncols, double *out) {
    __shared__ double red[8][32];
    const int warp = threadIdx.x >> 5, ln = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int c0 = 0; c0 < ncols; c0 += 8) {
        double acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = 0.0;
#pragma unroll 4
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (c0 + q < ncols) acc[q] += __ldcg(partial + (long long)(c0 + q) * nb + b);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const double v = warp_sum(acc[q]);
            if (ln == 0) red[q][warp] = v;
        }
        __syncthreads();
        if ((int)threadIdx.x < 8 && c0 + (int)threadIdx.x < ncols) {
            double u = 0.0;
            for (int w = 0; w < nw; ++w) u += red[threadIdx.x][w];
            out[c0 + threadIdx.x] = u;
        }
        __syncthreads();
    }
}

// out[col] = sum_b of the float-float partials of column col: warp w takes
// columns w, w + 8, ...; lane l adds partials b = l, l + 32, ... in ascending
// order, then a fixed warp tree (one order whatever the scheduling).
__device__ __forceinline__ void block_reduce_partials_ff(const double *partial, int nb, int ncols, double *out) {
    const int warp = threadIdx.x >> 5, ln = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int col = warp; col < ncols; col += nw) {
        const float2 *p = reinterpret_cast<const float2 *>(partial + (long long)col * nb);
        FF a{0.f, 0.f};
#pragma unroll 4
        for (int b = ln; b < nb; b += 32) {
            const float2 v = __ldcg(p + b);
            a = ff_add(a, FF{v.x, v.y});
        }
        a = ff_warp_sum(a);
        if (ln == 0) out[col] = ff_to_double(a);
    }
}
// the last block's reduction of a T kernel's partials
template <typename T> __device__ __forceinline__ void reduce_partials(const double *partial, int nb, int ncols, double *out) {
    if constexpr (std::is_same<T, float>::value) block_reduce_partials_ff(partial, nb, ncols, out);
    else block_reduce_partials(partial, nb, ncols, out);
}

// Block stage of the grid reductions: for q < nq, the sum of acc[q] over the
// block's threads into partial[(col0 + q) * gridDim.x + blockIdx.x].  FP64
// kernels: FP64 warp trees, then the warps' sums in order; FP32 kernels: the
// same in float-float (the partial stored as a float2).  256 threads.
template <typename T, int NQ>
__device__ __forceinline__ void block_partials(const T (&acc)[NQ], int nq, double *partial, int col0) {
    const int warp = threadIdx.x >> 5, ln = threadIdx.x & 31, nw = blockDim.x >> 5;
    if constexpr (std::is_same<T, float>::value) {
        __shared__ FF redf[NQ][8];
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            if (q < nq) {   // uniform over the block
                const FF v = ff_warp_sum(FF{acc[q], 0.f});
                if (ln == 0) redf[q][warp] = v;
            }
        __syncthreads();
        if ((int)threadIdx.x < nq) {
            FF u = redf[threadIdx.x][0];
            for (int k = 1; k < nw; ++k) u = ff_add(u, redf[threadIdx.x][k]);
            *reinterpret_cast<float2 *>(partial + (long long)(col0 + threadIdx.x) * gridDim.x + blockIdx.x) =
                make_float2(u.hi, u.lo);
        }
    } else {
        __shared__ double redd[NQ][8];
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            if (q < nq) {
                const double v = warp_sum((double)acc[q]);
                if (ln == 0) redd[q][warp] = v;
            }
        __syncthreads();
        if ((int)threadIdx.x < nq) {
            double u = 0.0;
            for (int k = 0; k < nw; ++k) u += redd[threadIdx.x][k];
            partial[(long long)(col0 + threadIdx.x) * gridDim.x + blockIdx.x] = u;
        }
    }
}

// Scalar-block (Ŝ level) sliced-ELL product y = M x fused with the inner
// products the K-cycle takes of it: kd[o0] = y . da and, when db is set,
// kd[o1] = y . db (da may be y itself).  T threads per row as in k_sellm
// (T = 1: one thread per row); each row's sum is the same as the unfused
// kernels'.  The row products are summed per warp in FP64, per block in a
// fixed order into part[b] and part[nb + b], and the last block to finish
// (ticket kd[7]) adds the block partials in a fixed order -- one launch
// instead of a product and a reduction, the same result whatever the order
// the blocks run in.
struct DotArgs {
    const void *da, *db;   // vectors the product is dotted with (same type as y); db may be null
    double *part;          // 2 x gridDim.x block partials
    double *kd;            // results kd[o0], kd[o1]; kd[7] is the ticket
    int o0, o1;
};
template <typename VT, typename XT, int C, int T>
__global__ void __launch_bounds__(256) k_sell_dot(SpmvArgs a, DotArgs q) {
    using AT = XT;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int row = (int)(gid / T), h = (int)(gid % T);
    const int sl = row / C, t = row % C;
    const bool live = sl < a.nslice;
    const long long base = live ? a.sl_ptr[sl] : 0;
    const int w = live ? (int)((a.sl_ptr[sl + 1] - base) / C) : 0;
    const VT *__restrict__ val = (const VT *)a.val;
    const XT *__restrict__ x = (const XT *)a.x;
    AT acc0 = 0, acc1 = 0, acc2 = 0;
    if constexpr (std::is_same<VT, __nv_bfloat16>::value) {
        sell_pairs<1, C>(a, base / 2, w / 2, t, h, T, x, acc0, acc1, acc2);
        if ((w & 1) && h == (w / 2) % T) sell_single<1, C>(a, base + (long long)C * (w - 1), t, x, acc0, acc1, acc2);
    } else {
        for (int k = h; k < w; k += T) {
            const long long g = base + (long long)C * k;
            acc0 += cvt<AT>(ldm<C == 32>(val + g + t)) * __ldg(x + ldm<C == 32>(a.sl_ci + g + t));
        }
    }
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) acc0 += __shfl_xor_sync(0xffffffffu, acc0, o);
    AT p0 = 0, p1 = 0;
    if (h == 0 && live && row < a.nbr) {
        ((XT *)a.y)[row] = acc0;
        p0 = acc0 * (q.da == a.y ? acc0 : ((const XT *)q.da)[row]);
        if (q.db) p1 = acc0 * ((const XT *)q.db)[row];
    }
    const AT pp[2] = {p0, p1};
    block_partials<AT, 2>(pp, 2, q.part, 0);
    unsigned *ticket = (unsigned *)(q.kd + 7);
    if (!grid_last_block(ticket)) return;
    __shared__ double out[2];
    reduce_partials<AT>(q.part, gridDim.x, q.db ? 2 : 1, out);
    __syncthreads();
    if (threadIdx.x == 0) {
        q.kd[q.o0] = out[0];
        if (q.db) q.kd[q.o1] = out[1];
        *ticket = 0;
    }
}

// ================================================ Givens / least squares
struct GmState {
    double res;      // |g_{j+1}|
    double beta;     // h_{j+1,j}
    int nan;         // NaN/Inf met
    int pad;
};

// What the fused Givens update of Hessenberg column j needs (H == nullptr:
// no update).
struct GivensArgs {
    double *H = nullptr;
    int ldh = 0, j = 0;
    const int *jp = nullptr;   // when set, the column index is read here (device-driven loops)
    const double *h1 = nullptr, *h2 = nullptr;
    double *cs = nullptr, *sn = nullptr, *g = nullptr;
    GmState *st = nullptr;
};

// Column j of the Hessenberg matrix: H(i,j) = h1_i + h2_i (i <= j; h1_i
// alone when h2 is null, a single Gram-Schmidt pass),
// H(j+1,j) = ||w|| (from ||w||^2 = nrm2); the previous rotations applied, a
// new rotation chosen to zero H(j+1,j), and the right-hand side g rotated
// (Saad 1993, FGMRES with Givens rotations).  One thread.
__device__ __forceinline__ void givens_step(const GivensArgs &q, double nrm2) {
    double *H = q.H;
    const long long ldh = q.ldh;
    const int j = q.jp ? *q.jp : q.j;
    for (int i = 0; i <= j; ++i) H[i * ldh + j] = q.h2 ? q.h1[i] + q.h2[i] : q.h1[i];
    const double beta = (nrm2 >= 0.0) ? sqrt(nrm2) : nrm2;   // NaN passes through
    H[(j + 1) * ldh + j] = beta;
    for (int i = 0; i < j; ++i) {
        const double a = H[i * ldh + j], b = H[(i + 1) * ldh + j];
        H[i * ldh + j] = q.cs[i] * a + q.sn[i] * b;
        H[(i + 1) * ldh + j] = -q.sn[i] * a + q.cs[i] * b;
    }
    const double a = H[j * ldh + j], b = H[(j + 1) * ldh + j];
    const double den = hypot(a, b);
    if (den == 0.0) { q.cs[j] = 1.0; q.sn[j] = 0.0; }
    else { q.cs[j] = a / den; q.sn[j] = b / den; }
    H[j * ldh + j] = den;
    H[(j + 1) * ldh + j] = 0.0;
    q.g[j + 1] = -q.sn[j] * q.g[j];
    q.g[j] = q.cs[j] * q.g[j];
    const double res = fabs(q.g[j + 1]);
    q.st->res = res;
    q.st->beta = beta;
    q.st->nan = (isfinite(res) && isfinite(beta)) ? 0 : 1;
}

// out[c] = V(:, c)^T w for c < ncols (column c at V + c*ldv), over the fixed
// grid; VEC: every pointer and ldv are 16-byte aligned.  When gv.H is set
// (ncols == 1, w the new Arnoldi vector) the last block also applies the
// Givens update with out[0] = ||w||^2.
template <typename T, int CB, bool VEC>
__device__ __forceinline__ void mdot_body(const T *__restrict__ V, long long ldv, int ncols, const T *__restrict__ w,
                                          long long n, double *__restrict__ partial, double *__restrict__ out,
                                          unsigned *ticket, const GivensArgs &gv) {
    constexpr int W = VEC ? Vec16<T>::W : 1;
    long long lo, hi;
    block_chunk(n, Vec16<T>::W, lo, hi);
    const long long nv = (hi - lo) / W;
    for (int c0 = 0; c0 < ncols; c0 += CB) {
        T acc[CB];
#pragma unroll
        for (int q = 0; q < CB; ++q) acc[q] = 0;
        for (long long i = threadIdx.x; i < nv; i += blockDim.x) {
            const long long t = lo + i * W;
            if constexpr (VEC) {
                T wt[W];
                vld(w + t, wt);
#pragma unroll
                for (int q = 0; q < CB; ++q)
                    if (c0 + q < ncols) {
                        T v[W];
                        vld(V + (long long)(c0 + q) * ldv + t, v);
#pragma unroll
                        for (int e = 0; e < W; ++e) acc[q] += v[e] * wt[e];
                    }
            } else {
                const T wt = w[t];
#pragma unroll
                for (int q = 0; q < CB; ++q)
                    if (c0 + q < ncols) acc[q] += V[(long long)(c0 + q) * ldv + t] * wt;
            }
        }
        if (VEC && threadIdx.x < hi - lo - nv * W) {   // ragged end of the last chunk
            const long long t = lo + nv * W + threadIdx.x;
            const T wt = w[t];
#pragma unroll
            for (int q = 0; q < CB; ++q)
                if (c0 + q < ncols) acc[q] += V[(long long)(c0 + q) * ldv + t] * wt;
        }
        block_partials<T, CB>(acc, min(CB, ncols - c0), partial, c0);
        __syncthreads();
    }
    if (!grid_last_block(ticket)) return;
    reduce_partials<T>(partial, gridDim.x, ncols, out);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (gv.H) givens_step(gv, out[0]);
        *ticket = 0;
    }
}

template <typename T, int CB, bool VEC>
__global__ void __launch_bounds__(256) k_mdot(const T *__restrict__ V, long long ldv, int ncols, const T *__restrict__ w,
                                              long long n, double *__restrict__ partial, double *__restrict__ out,
                                              unsigned *ticket, GivensArgs gv) {
    mdot_body<T, CB, VEC>(V, ldv, ncols, w, n, partial, out, ticket, gv);
}
// the same with ncols = *jp + off read on the device (device-driven loops)
template <typename T, int CB, bool VEC>
__global__ void __launch_bounds__(256) k_mdot_dl(const T *__restrict__ V, long long ldv, const int *jp, int off,
                                                 const T *__restrict__ w, long long n, double *__restrict__ partial,
                                                 double *__restrict__ out, unsigned *ticket, GivensArgs gv) {
    mdot_body<T, CB, VEC>(V, ldv, *jp + off, w, n, partial, out, ticket, gv);
}

// w[t] += alpha * sum_j coef[j] V[j][t]  (coef on the device, FP64)
template <typename T, bool VEC>
__device__ __forceinline__ void maxpy_body(const T *__restrict__ V, long long ldv, int ncols, const double *__restrict__ coef,
                                           double alpha, T *__restrict__ w, long long n) {
    constexpr int W = VEC ? Vec16<T>::W : 1;
    __shared__ T cs[256];
    const long long nv = n / W;
    for (int c0 = 0; c0 < ncols; c0 += 256) {
        const int cn = min(256, ncols - c0);
        __syncthreads();
        if ((int)threadIdx.x < cn) cs[threadIdx.x] = (T)(alpha * coef[c0 + threadIdx.x]);
        __syncthreads();
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (long long)gridDim.x * blockDim.x) {
            const long long t = i * W;
            T acc[W];
            if constexpr (VEC) vld(w + t, acc);
            else acc[0] = w[t];
            for (int j = 0; j < cn; ++j) {
                T v[W];
                if constexpr (VEC) vld(V + (long long)(c0 + j) * ldv + t, v);
                else v[0] = V[(long long)(c0 + j) * ldv + t];
#pragma unroll
                for (int e = 0; e < W; ++e) acc[e] += cs[j] * v[e];
            }
            if constexpr (VEC) vst(w + t, acc);
            else w[t] = acc[0];
        }
        if (VEC && blockIdx.x == 0 && threadIdx.x < n - nv * W) {   // ragged end
            const long long t = nv * W + threadIdx.x;
            T acc = w[t];
            for (int j = 0; j < cn; ++j) acc += cs[j] * V[(long long)(c0 + j) * ldv + t];
            w[t] = acc;
        }
    }
}

template <typename T, bool VEC>
__global__ void __launch_bounds__(256) k_maxpy(const T *__restrict__ V, long long ldv, int ncols, const double *__restrict__ coef,
                                               double alpha, T *__restrict__ w, long long n) {
    maxpy_body<T, VEC>(V, ldv, ncols, coef, alpha, w, n);
}
template <typename T, bool VEC>
__global__ void __launch_bounds__(256) k_maxpy_dl(const T *__restrict__ V, long long ldv, const int *jp, int off,
                                                  const double *__restrict__ coef, double alpha, T *__restrict__ w,
                                                  long long n) {
    maxpy_body<T, VEC>(V, ldv, *jp + off, coef, alpha, w, n);
}

// Fused CGS pass for up to MAXC columns: w_new = w - sum_j coef[j] V[j], then
// the dots of the same columns with w_new (norm_only = 0) or the squared norm
// of w_new (norm_only = 1), V read once; partials reduced by the last block
// into out (and, with gv.H set, the Givens update with out[0] = ||w_new||^2).
template <typename T, int MAXC, bool VEC>
__device__ __forceinline__ void maxpy_dot_body(const T *__restrict__ V, long long ldv, int ncols,
                                               const double *__restrict__ coef, T *__restrict__ w, long long n,
                                               int norm_only, double *__restrict__ partial, double *__restrict__ out,
                                               unsigned *ticket, const GivensArgs &gv) {
    constexpr int W = VEC ? Vec16<T>::W : 1;
    __shared__ T cs[MAXC];
    if ((int)threadIdx.x < ncols) cs[threadIdx.x] = (T)coef[threadIdx.x];
    __syncthreads();
    long long lo, hi;
    block_chunk(n, Vec16<T>::W, lo, hi);
    const long long nv = (hi - lo) / W;
    T acc[MAXC];
#pragma unroll
    for (int q = 0; q < MAXC; ++q) acc[q] = 0;
    auto body = [&](long long t, auto wtag) {
        constexpr int L = decltype(wtag)::value;
        T v[MAXC][L], s[L];
        if constexpr (L > 1) vld(w + t, s);
        else s[0] = w[t];
#pragma unroll
        for (int q = 0; q < MAXC; ++q)
            if (q < ncols) {
                if constexpr (L > 1) vld(V + (long long)q * ldv + t, v[q]);
                else v[q][0] = V[(long long)q * ldv + t];
#pragma unroll
                for (int e = 0; e < L; ++e) s[e] -= cs[q] * v[q][e];
            }
        if constexpr (L > 1) vst(w + t, s);
        else w[t] = s[0];
        if (norm_only) {
#pragma unroll
            for (int e = 0; e < L; ++e) acc[0] += s[e] * s[e];
        } else {
#pragma unroll
            for (int q = 0; q < MAXC; ++q)
                if (q < ncols) {
#pragma unroll
                    for (int e = 0; e < L; ++e) acc[q] += v[q][e] * s[e];
                }
        }
    };
    for (long long i = threadIdx.x; i < nv; i += blockDim.x) body(lo + i * W, std::integral_constant<int, W>());
    if (VEC && threadIdx.x < hi - lo - nv * W) body(lo + nv * W + threadIdx.x, std::integral_constant<int, 1>());
    const int nout = norm_only ? 1 : ncols;
    block_partials<T, MAXC>(acc, nout, partial, 0);
    if (!grid_last_block(ticket)) return;
    reduce_partials<T>(partial, gridDim.x, nout, out);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (gv.H) givens_step(gv, out[0]);
        *ticket = 0;
    }
}

template <typename T, int MAXC, bool VEC>
__global__ void __launch_bounds__(256) k_maxpy_dot(const T *__restrict__ V, long long ldv, int ncols,
                                                   const double *__restrict__ coef, T *__restrict__ w, long long n,
                                                   int norm_only, double *__restrict__ partial, double *__restrict__ out,
                                                   unsigned *ticket, GivensArgs gv) {
    maxpy_dot_body<T, MAXC, VEC>(V, ldv, ncols, coef, w, n, norm_only, partial, out, ticket, gv);
}

// The device-driven form of the fused pass, ncols = *jp + off read on the
// device.  A basis longer than MAXC takes two sweeps over the block's own
// chunk: the subtraction w -= V coef (columns in ascending order, each
// thread on the elements it owns), then mdot_body's products (or norm and
// Givens update) on the same elements, so no element crosses threads.
template <typename T, int MAXC, bool VEC>
__global__ void __launch_bounds__(256) k_maxpy_dot_dl(const T *__restrict__ V, long long ldv, const int *jp, int off,
                                                      const double *__restrict__ coef, T *__restrict__ w, long long n,
                                                      int norm_only, double *__restrict__ partial,
                                                      double *__restrict__ out, unsigned *ticket, GivensArgs gv) {
    const int ncols = *jp + off;
    if (ncols <= MAXC) {
        maxpy_dot_body<T, MAXC, VEC>(V, ldv, ncols, coef, w, n, norm_only, partial, out, ticket, gv);
        return;
    }
    constexpr int W = VEC ? Vec16<T>::W : 1;
    __shared__ T cs[256];
    long long lo, hi;
    block_chunk(n, Vec16<T>::W, lo, hi);
    const long long nv = (hi - lo) / W;
    for (int c0 = 0; c0 < ncols; c0 += 256) {
        const int cn = min(256, ncols - c0);
        __syncthreads();
        if ((int)threadIdx.x < cn) cs[threadIdx.x] = (T)coef[c0 + threadIdx.x];
        __syncthreads();
        for (long long i = threadIdx.x; i < nv; i += blockDim.x) {
            const long long t = lo + i * W;
            T a[W];
            if constexpr (VEC) vld(w + t, a);
            else a[0] = w[t];
            for (int j = 0; j < cn; ++j) {
                T v[W];
                if constexpr (VEC) vld(V + (long long)(c0 + j) * ldv + t, v);
                else v[0] = V[(long long)(c0 + j) * ldv + t];
#pragma unroll
                for (int e = 0; e < W; ++e) a[e] -= cs[j] * v[e];
            }
            if constexpr (VEC) vst(w + t, a);
            else w[t] = a[0];
        }
        if (VEC && threadIdx.x < hi - lo - nv * W) {   // ragged end, the thread mdot_body gives it
            const long long t = lo + nv * W + threadIdx.x;
            T a = w[t];
            for (int j = 0; j < cn; ++j) a -= cs[j] * V[(long long)(c0 + j) * ldv + t];
            w[t] = a;
        }
    }
    __syncthreads();
    if (norm_only) mdot_body<T, 8, VEC>(w, ldv, 1, w, n, partial, out, ticket, gv);
    else mdot_body<T, 8, VEC>(V, ldv, ncols, w, n, partial, out, ticket, gv);
}

// ============================================================== vectors
template <typename T> __global__ void k_fill(T *x, T v, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) x[i] = v;
}
template <typename D, typename S> __global__ void k_convert(D *dst, const S *src, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = (D)src[i];
}
// y = a*x + b*y
template <typename T> __global__ void k_axpby(T *y, const T *x, double a, double b, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = (T)a * x[i] + (T)b * y[i];
}
// z = x - y
template <typename T> __global__ void k_sub(T *z, const T *x, const T *y, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        z[i] = x[i] - y[i];
}
// v = w / s[0] (skips when s[0] == 0); VEC: v, w 16-byte aligned
template <typename T, bool VEC> __device__ __forceinline__ void scale_inv_body(T *v, const T *w, const double *s, long long n) {
    constexpr int W = VEC ? Vec16<T>::W : 1;
    __shared__ T inv_s;
    __shared__ int zero;
    if (threadIdx.x == 0) {   // one FP64 division per block, not per element
        const double d = *s;
        zero = (d == 0.0);
        inv_s = zero ? T(0) : (T)(1.0 / d);
    }
    __syncthreads();
    if (zero) return;
    const T inv = inv_s;
    const long long nv = n / W;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (long long)gridDim.x * blockDim.x) {
        if constexpr (VEC) {
            T u[W];
            vld(w + i * W, u);
#pragma unroll
            for (int e = 0; e < W; ++e) u[e] *= inv;
            vst(v + i * W, u);
        } else {
            v[i] = w[i] * inv;
        }
    }
    if (VEC && blockIdx.x == 0 && threadIdx.x < n - nv * W) v[nv * W + threadIdx.x] = w[nv * W + threadIdx.x] * inv;
}
template <typename T, bool VEC> __global__ void k_scale_inv(T *v, const T *w, const double *s, long long n) {
    scale_inv_body<T, VEC>(v, w, s, n);
}

// ============================================= least squares (GMRES end)
// y = H(0:k,0:k)^{-1} g(0:k), upper triangular.  One thread.
__global__ void k_trisolve(const double *H, int ldh, const double *g, double *y, int k);
// g = [beta, 0, ...]; st->res = beta
__global__ void k_gm_init(double *g, int m1, const double *beta2, double *beta, GmState *st);

__global__ void k_recip(long long n, const double *a, double *b);

// ============================== device-driven Krylov loops (graph WHILE)
// Loop state of one GMRES level on the device.
struct GmDev {
    int j, its, m, nmax;        // column of the current cycle, iterations, restart length, iteration limit
    int conv, nan, pad0, pad1;  // pad0: restart cycles run (outer level)
    double tol, bnorm, res, rel_true;
};
// Per-solve options of the device-driven solve (written before each launch).
struct DlParams {
    double rtol, rtol_A, rtol_S, rtol_I, atol;
    int m, m_A, m_S, nmax, nmax_A, nmax_S;
};
// Iteration counters of one device-driven solve.
struct DlCounters {
    long long A, S, I, nA, nS, nI;
};
__global__ void k_dl_init(GmDev *st, double *g, int m1, const double *nrm2, double *beta, GmState *gs,
                          const double *rtol, const double *atol, const int *m, const int *nmax,
                          cudaGraphConditionalHandle h);
// The end of one iteration of a device-driven GMRES loop (one thread):
// counters, then the stopping rule of the host-driven loop -- continue while
// |g_{j+1}| > max(rtol ||b||, atol), h_{j+1,j} != 0, no NaN, j < m and
// its < n_max -- as the WHILE node's condition.
__device__ __forceinline__ void dl_step(GmDev *st, const GmState *gs, cudaGraphConditionalHandle h) {
    st->its += 1;
    st->j += 1;
    st->res = gs->res;
    if (gs->nan) st->nan = 1;
    const bool go = !st->nan && st->res > st->tol && gs->beta != 0.0 && st->j < st->m && st->its < st->nmax;
    cudaGraphSetConditional(h, go ? 1u : 0u);
}
// The last kernel of an iteration: basis column j + 1 = w / h_{j+1,j}
// (gs->beta, the reciprocal taken once per block as in k_scale_inv), then,
// in the grid's last block -- every block has read j by then -- dl_step.
template <typename T, bool VEC>
__global__ void k_scale_step_dl(T *vbase, long long ld, GmDev *st, const T *w, const GmState *gs, long long n,
                                unsigned *ticket, cudaGraphConditionalHandle h) {
    constexpr int W = VEC ? Vec16<T>::W : 1;
    __shared__ T inv_s;
    __shared__ int zero;
    if (threadIdx.x == 0) {
        const double d = gs->beta;
        zero = (d == 0.0);
        inv_s = zero ? T(0) : (T)(1.0 / d);
    }
    __syncthreads();
    T *v = vbase + (long long)(st->j + 1) * ld;
    if (!zero) {
        const T inv = inv_s;
        const long long nv = n / W;
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (long long)gridDim.x * blockDim.x) {
            if constexpr (VEC) {
                T u[W];
                vld(w + i * W, u);
#pragma unroll
                for (int e = 0; e < W; ++e) u[e] *= inv;
                vst(v + i * W, u);
            } else {
                v[i] = w[i] * inv;
            }
        }
        if (VEC && blockIdx.x == 0 && threadIdx.x < n - nv * W) v[nv * W + threadIdx.x] = w[nv * W + threadIdx.x] * inv;
    }
    if (!grid_last_block(ticket)) return;
    if (threadIdx.x == 0) {
        dl_step(st, gs, h);
        *ticket = 0;
    }
}
__global__ void k_dl_cycle_start(GmDev *st, cudaGraphConditionalHandle h);
__global__ void k_dl_end(GmDev *st, const double *H, int ldh, const double *g, double *y, long long *its_total,
                         long long *solves);
__global__ void k_dl_restart(GmDev *st, const double *nrm2, double *g, int m1, double *beta, GmState *gs,
                             cudaGraphConditionalHandle h);

// out = entries [from, from + n) of basis column *jp + off (stride ld), converted
template <typename D, typename S>
__global__ void k_col_get(D *out, const S *vbase, long long ld, const int *jp, int off, long long from, long long n) {
    const S *v = vbase + (long long)(*jp + off) * ld + from;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (D)v[i];
}
// entries [to, to + n) of basis column *jp + off = in, converted
template <typename D, typename S>
__global__ void k_col_put(D *vbase, long long ld, const int *jp, int off, long long to, const S *in, long long n) {
    D *v = vbase + (long long)(*jp + off) * ld + to;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v[i] = (D)in[i];
}
// out = x .* d with x basis column *jp (point Jacobi from a column)
template <typename T>
__global__ void k_mul_col(T *out, const T *vbase, long long ld, const int *jp, const T *d, long long n) {
    const T *x = vbase + (long long)(*jp) * ld;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = x[i] * d[i];
}

// ================================================================= AMG
// coarse r_c[I] = sum_{i in I} r[i], bs components: 8 lanes per aggregate
// (aggregates have at most 8 members), member loads in parallel, then a
// fixed xor-shuffle tree inside the 8 lanes
template <typename T>
__global__ void k_restrict(const int *__restrict__ mptr, const int *__restrict__ mem, int nc, int bs, const T *__restrict__ r,
                           T *__restrict__ rc) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int I = (int)(g >> 3), l = (int)(g & 7);
    const bool live = I < nc;
    const unsigned mask = 0xffu << (threadIdx.x & 24u);
    if (__all_sync(0xffffffffu, !live)) return;   // whole warp past the end
    int q = 0, beg = 0;
    if (live) { beg = mptr[I]; q = mptr[I + 1] - beg; }
    const int m = (live && l < q) ? mem[beg + l] : -1;
    for (int a = 0; a < bs; ++a) {
        T s = (m >= 0) ? r[(long long)m * bs + a] : T(0);
        s += __shfl_xor_sync(mask, s, 4);
        s += __shfl_xor_sync(mask, s, 2);
        s += __shfl_xor_sync(mask, s, 1);
        if (live && l == 0) rc[(long long)I * bs + a] = s;
    }
}
// Restriction fused with the first Chebyshev step of the coarse level's
// pre-smoothing (which starts from zero): rc = R r, then d = c2 Dinv_c rc and
// x = d, as k_restrict followed by k_cheb_first on the coarse level computes
// them (same operations, same order); rcopy (optional) gets a copy of rc.
template <typename T>
__global__ void k_restrict_first(const int *__restrict__ mptr, const int *__restrict__ mem, int nc, int bs,
                                 const T *__restrict__ r, T *__restrict__ rc, const T *__restrict__ dinv, T c2,
                                 T *__restrict__ d, T *__restrict__ x, T *__restrict__ rcopy) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int I = (int)(g >> 3), l = (int)(g & 7);
    const bool live = I < nc;
    const unsigned mask = 0xffu << (threadIdx.x & 24u);
    if (__all_sync(0xffffffffu, !live)) return;
    int q = 0, beg = 0;
    if (live) { beg = mptr[I]; q = mptr[I + 1] - beg; }
    const int m = (live && l < q) ? mem[beg + l] : -1;
    T v[3] = {T(0), T(0), T(0)};   // bs <= 3; every lane of the group ends with the sums
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a < bs) {
            T s = (m >= 0) ? r[(long long)m * bs + a] : T(0);
            s += __shfl_xor_sync(mask, s, 4);
            s += __shfl_xor_sync(mask, s, 2);
            s += __shfl_xor_sync(mask, s, 1);
            v[a] = s;
        }
    }
    if (!live || l >= bs) return;
    // lane l < bs finishes component l of aggregate I
    const long long t = (long long)I * bs + l;
    const T vl = (l == 0) ? v[0] : (l == 1) ? v[1] : v[2];
    rc[t] = vl;
    if (rcopy) rcopy[t] = vl;
    T s = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c)
        if (c < bs) s += dinv[(long long)I * bs * bs + l * bs + c] * v[c];
    const T dn = c2 * s;
    d[t] = dn;
    x[t] = dn;
}
// x[i] += e_c[agg[i]]
template <typename T>
__global__ void k_prolong(const int *__restrict__ agg, int n, int bs, const T *__restrict__ ec, T *__restrict__ x) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * bs) return;
    const int i = (int)(t / bs), a = (int)(t - (long long)i * bs);
    const int I = agg[i];
    if (I >= 0) x[t] += ec[(long long)I * bs + a];
}
// The same for blocks of BS components with W = Vec16<T>::W consecutive
// nodes per thread: their map entries and BS 16-byte pieces of x loaded at
// once (the one-component form keeps a single load chain per thread), the
// same per-element adds; the last n % W nodes one per thread.  x and agg
// 16-byte aligned.
template <typename T, int BS>
__global__ void k_prolong_v(const int *__restrict__ agg, int n, const T *__restrict__ ec, T *__restrict__ x) {
    constexpr int W = Vec16<T>::W;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long ng = n / W;
    if (g < ng) {
        int I[W];
#pragma unroll
        for (int e = 0; e < W; ++e) I[e] = agg[g * W + e];
        T v[BS][W];
#pragma unroll
        for (int c = 0; c < BS; ++c) vld(x + (g * BS + c) * W, v[c]);
#pragma unroll
        for (int k = 0; k < BS * W; ++k) {   // element k: node k / BS, component k % BS
            const int Ik = I[k / BS];
            if (Ik >= 0) v[k / W][k % W] += ec[(long long)Ik * BS + k % BS];
        }
#pragma unroll
        for (int c = 0; c < BS; ++c) vst(x + (g * BS + c) * W, v[c]);
    } else if (g < ng + n % W) {
        const long long i = ng * W + (g - ng);
        const int Ii = agg[i];
        if (Ii >= 0) {
#pragma unroll
            for (int a = 0; a < BS; ++a) x[i * BS + a] += ec[(long long)Ii * BS + a];
        }
    }
}
// Chebyshev first step from x = 0: d = c2 Dinv b; x = d
// (bcopy != nullptr: b is also copied there, for a cycle replayed on fixed buffers)
template <typename T>
__global__ void k_cheb_first(int nbr, int bs, const T *__restrict__ dinv, const T *__restrict__ b, T c2, T *__restrict__ d,
                             T *__restrict__ x, T *__restrict__ bcopy) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)nbr * bs) return;
    if (bcopy) bcopy[t] = b[t];
    const int i = (int)(t / bs), a = (int)(t - (long long)i * bs);
    T s = 0;
    for (int c = 0; c < bs; ++c) s += dinv[(long long)i * bs * bs + a * bs + c] * b[(long long)i * bs + c];
    const T dn = c2 * s;
    d[t] = dn;
    x[t] = dn;
}
// k_cheb_first with b = basis column *jp (stride ld)
template <typename T>
__global__ void k_cheb_first_col(int nbr, int bs, const T *__restrict__ dinv, const T *__restrict__ vbase, long long ld,
                                 const int *jp, T c2, T *__restrict__ d, T *__restrict__ x, T *__restrict__ bcopy) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)nbr * bs) return;
    const T *b = vbase + (long long)(*jp) * ld;
    if (bcopy) bcopy[t] = b[t];
    const int i = (int)(t / bs), a = (int)(t - (long long)i * bs);
    T s = 0;
    for (int c = 0; c < bs; ++c) s += dinv[(long long)i * bs * bs + a * bs + c] * b[(long long)i * bs + c];
    const T dn = c2 * s;
    d[t] = dn;
    x[t] = dn;
}
// x = Cinv b, dense (coarsest level); one warp per row; the inverse is stored
// in the vector type (FP64 or FP32).  Each lane keeps four independent
// partial sums and, when rows start on 16-byte boundaries, reads 16 bytes
// at a time, so a lane has several loads in flight instead of one long
// chain of dependent adds; the partials are added in a fixed order.
template <typename T>
__global__ void k_dense_gemv(const T *__restrict__ Cinv, int n, const T *__restrict__ b, T *__restrict__ x) {
    constexpr int W = Vec16<T>::W;
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int ln = threadIdx.x & 31;
    if (row >= n) return;
    const T *r = Cinv + (long long)row * n;
    T s[4] = {0, 0, 0, 0};
    if (n % W == 0 && ((uintptr_t)Cinv & 15u) == 0 && ((uintptr_t)b & 15u) == 0) {
        const int nv = n / W;
#pragma unroll 4
        for (int c = ln; c < nv; c += 32) {
            T a[W], v[W];
            vld(r + (long long)c * W, a);
            vld(b + (long long)c * W, v);
#pragma unroll
            for (int e = 0; e < W; ++e) s[e % 4] += a[e] * v[e];
        }
    } else {
        int c = ln;
        for (; c + 96 < n; c += 128) {
#pragma unroll
            for (int q = 0; q < 4; ++q) s[q] += r[c + 32 * q] * b[c + 32 * q];
        }
        for (; c < n; c += 32) s[0] += r[c] * b[c];
    }
    T t = (s[0] + s[1]) + (s[2] + s[3]);
    t = warp_sum(t);
    if (ln == 0) x[row] = t;
}

// The FP32 form with a block of kGemvThreads threads (four warps) per row:
// each thread keeps four partial sums over the 16-byte pieces t, t + 128, ...
// of the row, then a fixed warp tree per warp and the four warps' sums in
// order.  A row of a coarsest inverse about 1300 wide is about 330 pieces,
// three per thread, so a row's loads are in flight together instead of ten
// deep in one warp.  VEC: rows on 16-byte boundaries (n % 4 == 0, Cinv and b
// aligned); otherwise single floats c = t, t + 128, ... into the four sums in
// turn.
constexpr int kGemvThreads = 128;
template <typename T, bool VEC>   // float
__global__ void __launch_bounds__(kGemvThreads) k_dense_gemv_rows(const T *__restrict__ Cinv, int n,
                                                                  const T *__restrict__ b, T *__restrict__ x) {
    static_assert(std::is_same<T, float>::value, "FP32 form");
    __shared__ float ws[kGemvThreads / 32];
    const int row = blockIdx.x;
    const float *r = Cinv + (long long)row * n;
    float s[4] = {0.f, 0.f, 0.f, 0.f};
    if constexpr (VEC) {
        const int nv = n / 4;
        for (int c = threadIdx.x; c < nv; c += kGemvThreads) {
            float a[4], v[4];
            vld(r + (long long)c * 4, a);
            vld(b + (long long)c * 4, v);
#pragma unroll
            for (int e = 0; e < 4; ++e) s[e] += a[e] * v[e];
        }
    } else {
        int c = threadIdx.x;
        for (; c + 3 * kGemvThreads < n; c += 4 * kGemvThreads) {
#pragma unroll
            for (int e = 0; e < 4; ++e) s[e] += r[c + e * kGemvThreads] * b[c + e * kGemvThreads];
        }
        for (int e = 0; c < n; c += kGemvThreads, ++e) s[e] += r[c] * b[c];
    }
    float t = (s[0] + s[1]) + (s[2] + s[3]);
    t = warp_sum(t);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        float u = ws[0];
#pragma unroll
        for (int w = 1; w < kGemvThreads / 32; ++w) u += ws[w];
        x[row] = u;
    }
}

// ============================================================== K-cycle
// kd[o0] = a.b and, when c != nullptr, kd[o1] = c.d.  Each block reduces a
// fixed contiguous chunk into kd[8 + 2 blk], and the last block to finish
// (ticket in kd[7]) sums the block partials in a fixed order (one warp,
// lanes over blocks): one launch, same result whatever order the blocks run in.
constexpr int kKdotBlocks = 96;

// The two sums p0, p1 of every thread reduced over the grid: per block into
// kd[8 + 2 blk], kd[9 + 2 blk], then by warp 0 of the last block to finish
// (ticket kd[7]; lanes over the blocks in steps of 32, a warp tree) into
// kd[o0] and, when two, kd[o1].  FP64 for FP64 vectors; float-float (float2
// in the slots) for FP32 ones.
template <typename T>
__device__ __forceinline__ void kdot_reduce(T p0, T p1, double *kd, int o0, int o1, bool two) {
    __shared__ bool last;
    if constexpr (std::is_same<T, float>::value) {
        __shared__ FF s0[8], s1[8];
        const FF t0 = ff_warp_sum(FF{p0, 0.f}), t1 = ff_warp_sum(FF{p1, 0.f});
        if ((threadIdx.x & 31) == 0) { s0[threadIdx.x >> 5] = t0; s1[threadIdx.x >> 5] = t1; }
        __syncthreads();
        if (threadIdx.x == 0) {
            FF u0 = s0[0], u1 = s1[0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) { u0 = ff_add(u0, s0[w]); u1 = ff_add(u1, s1[w]); }
            *reinterpret_cast<float2 *>(kd + 8 + 2 * blockIdx.x) = make_float2(u0.hi, u0.lo);
            *reinterpret_cast<float2 *>(kd + 9 + 2 * blockIdx.x) = make_float2(u1.hi, u1.lo);
            __threadfence();
            last = (atomicAdd((unsigned int *)(kd + 7), 1u) == gridDim.x - 1);
        }
        __syncthreads();
        if (last && threadIdx.x < 32) {
            __threadfence();
            FF u0{0.f, 0.f}, u1{0.f, 0.f};
            for (unsigned qb = threadIdx.x; qb < gridDim.x; qb += 32) {
                const float2 a0 = __ldcg(reinterpret_cast<const float2 *>(kd + 8 + 2 * qb));
                const float2 a1 = __ldcg(reinterpret_cast<const float2 *>(kd + 9 + 2 * qb));
                u0 = ff_add(u0, FF{a0.x, a0.y});
                u1 = ff_add(u1, FF{a1.x, a1.y});
            }
            u0 = ff_warp_sum(u0);
            u1 = ff_warp_sum(u1);
            if (threadIdx.x == 0) {
                kd[o0] = ff_to_double(u0);
                if (two) kd[o1] = ff_to_double(u1);
                *(unsigned int *)(kd + 7) = 0u;   // ready for the next call
            }
        }
    } else {
        __shared__ double s0[8], s1[8];
        const double t0 = warp_sum((double)p0), t1 = warp_sum((double)p1);
        if ((threadIdx.x & 31) == 0) { s0[threadIdx.x >> 5] = t0; s1[threadIdx.x >> 5] = t1; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double u0 = 0.0, u1 = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { u0 += s0[w]; u1 += s1[w]; }
            kd[8 + 2 * blockIdx.x] = u0;
            kd[9 + 2 * blockIdx.x] = u1;
            __threadfence();
            last = (atomicAdd((unsigned int *)(kd + 7), 1u) == gridDim.x - 1);
        }
        __syncthreads();
        if (last && threadIdx.x < 32) {
            __threadfence();
            double u0 = 0.0, u1 = 0.0;
            for (unsigned qb = threadIdx.x; qb < gridDim.x; qb += 32) {
                u0 += __ldcg(kd + 8 + 2 * qb);
                u1 += __ldcg(kd + 9 + 2 * qb);
            }
            u0 = warp_sum(u0);
            u1 = warp_sum(u1);
            if (threadIdx.x == 0) {
                kd[o0] = u0;
                if (two) kd[o1] = u1;
                *(unsigned int *)(kd + 7) = 0u;
            }
        }
    }
}
template <typename T>
__global__ void __launch_bounds__(256) k_kdots(const T *__restrict__ a, const T *__restrict__ b, const T *__restrict__ c,
                                               const T *__restrict__ d, long long n, double *kd, int o0, int o1) {
    const long long chunk = (n + gridDim.x - 1) / gridDim.x;
    const long long lo = (long long)blockIdx.x * chunk, hi = min(n, lo + chunk);
    T p0 = 0, p1 = 0;   // per-thread sums in the vector type
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        p0 += a[i] * b[i];
        if (c) p1 += c[i] * d[i];
    }
    kdot_reduce<T>(p0, p1, kd, o0, o1, c != nullptr);
}
// r -= a1 w1 with a1 = (w1.r)/(w1.w1) = kd[1]/kd[0]; a1 saved in kd[2]
template <typename T> __global__ void k_kupd1(T *r, const T *w1, double *kd, long long n) {
    __shared__ T a1s;
    if (threadIdx.x == 0) {
        const double a1 = kd[0] > 0.0 ? kd[1] / kd[0] : 0.0;
        a1s = (T)a1;
        if (blockIdx.x == 0) kd[2] = a1;
    }
    __syncthreads();
    const T a1 = a1s;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        r[i] = r[i] - a1 * w1[i];
}
// w2 -= beta w1 and z2 -= beta z1 with beta = (w2.w1)/(w1.w1) = kd[3]/kd[0],
// followed by kd[4] = w2.w2, kd[5] = w2.r on the updated w2, in one
// launch: the chunks, per-thread sums and fixed-order block and grid
// reductions of k_kdots (grid kKdotBlocks, ticket kd[7])
template <typename T>
__global__ void __launch_bounds__(256) k_kupd2_dots(T *__restrict__ w2, T *__restrict__ z2, const T *__restrict__ w1,
                                                    const T *__restrict__ z1, const T *__restrict__ r, double *kd,
                                                    long long n) {
    __shared__ T bs_;
    if (threadIdx.x == 0) bs_ = (T)(kd[0] > 0.0 ? kd[3] / kd[0] : 0.0);
    __syncthreads();
    const T beta = bs_;
    const long long chunk = (n + gridDim.x - 1) / gridDim.x;
    const long long lo = (long long)blockIdx.x * chunk, hi = min(n, lo + chunk);
    T p0 = 0, p1 = 0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const T wn = w2[i] - beta * w1[i];
        w2[i] = wn;
        z2[i] = z2[i] - beta * z1[i];
        p0 += wn * wn;
        p1 += wn * r[i];
    }
    kdot_reduce<T>(p0, p1, kd, 4, 5, true);
}
// x = a1 z1 + a2 z2 with a2 = (w2.r)/(w2.w2) = kd[5]/kd[4]
template <typename T> __global__ void k_kupd3(T *x, const T *z1, const T *z2, const double *kd, long long n) {
    __shared__ T a1s, a2s;
    if (threadIdx.x == 0) {
        a1s = (T)kd[2];
        a2s = (T)(kd[4] > 0.0 ? kd[5] / kd[4] : 0.0);
    }
    __syncthreads();
    const T a1 = a1s, a2 = a2s;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] = a1 * z1[i] + a2 * z2[i];
}

// =============================================================== rank one
// f[k] = r_k * (a^k . x), one block per outlet (fixed-order tree reduction)
template <typename T>
__global__ void k_lowrank_dots(const int *__restrict__ optr, const int *__restrict__ oidx, const double *__restrict__ oval,
                               const double *__restrict__ r, const T *__restrict__ x, double *__restrict__ f) {
    __shared__ double red[8];
    const int k = blockIdx.x;
    double s = 0.0;
    for (int q = optr[k] + threadIdx.x; q < optr[k + 1]; q += blockDim.x) s += oval[q] * (double)x[oidx[q]];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        f[k] = r[k] * t;
    }
}

}  // namespace nbp
