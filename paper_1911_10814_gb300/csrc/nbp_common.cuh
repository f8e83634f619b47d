// nbp_common.cuh -- shared device helpers and internal data structures of the
// GB300 nested block solver library (libnbp).  Internal header.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/nbp.h"

namespace nbp {

constexpr int kMaxLevels = 12;
constexpr int kSMs = 152;                 // GB300: 2 dies x 76 SMs
constexpr int kReduceBlocks = 4 * kSMs;   // fixed grid for deterministic reductions
constexpr int kCoarseDenseMax = 4096;     // largest coarsest level (scalar rows) solved densely

// ------------------------------------------------------------------ errors
struct Error {
    nbp_status st;
    std::string msg;
};

#define NBP_CUDA(call)                                                                        \
    do {                                                                                      \
        cudaError_t _e = (call);                                                              \
        if (_e != cudaSuccess) {                                                              \
            throw ::nbp::Error{_e == cudaErrorMemoryAllocation ? NBP_ERR_OOM : NBP_ERR_CUDA,  \
                               std::string(#call) + ": " + cudaGetErrorString(_e)};           \
        }                                                                                     \
    } while (0)

#define NBP_LAUNCHED()                                                                        \
    do {                                                                                      \
        cudaError_t _e = cudaGetLastError();                                                  \
        if (_e != cudaSuccess)                                                                \
            throw ::nbp::Error{NBP_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(_e)}; \
    } while (0)

inline void require(bool ok, nbp_status st, const std::string &msg) {
    if (!ok) throw Error{st, msg};
}

// --------------------------------------------------------------- numerics
template <typename T> struct Acc { using type = T; };
template <> struct Acc<__nv_bfloat16> { using type = float; };

__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ double to_d(float v) { return (double)v; }
__device__ __forceinline__ double to_d(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
__device__ __forceinline__ float to_f(double v) { return (float)v; }
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename A, typename V> __device__ __forceinline__ A cvt(V v);
template <> __device__ __forceinline__ double cvt<double, double>(double v) { return v; }
template <> __device__ __forceinline__ double cvt<double, float>(float v) { return (double)v; }
template <> __device__ __forceinline__ double cvt<double, __nv_bfloat16>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
template <> __device__ __forceinline__ float cvt<float, double>(double v) { return (float)v; }
template <> __device__ __forceinline__ float cvt<float, float>(float v) { return v; }
template <> __device__ __forceinline__ float cvt<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T> __device__ __forceinline__ T warp_sum(T v, unsigned mask = 0xffffffffu) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

// Float-float sums (the unevaluated sum hi + lo of two floats, about 44
// significant bits) for the reductions of the FP32 kernels.  GB300's FP64
// pipe retires about two operations per clock and SM (1.25 TFLOP/s for the
// GPU), so a tree of FP64 adds in every block's tail costs microseconds per
// block; these run on the FP32 pipe.  ff_add is Knuth's error-free two-sum of the leading parts, the
// trailing parts added to its error, then Dekker's fast two-sum to
// renormalise; all adds are explicitly rounded (no reassociation).
struct FF {
    float hi, lo;
};
__device__ __forceinline__ FF ff_add(FF a, FF b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float v = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float h = __fadd_rn(s, e);
    return FF{h, __fsub_rn(e, __fsub_rn(h, s))};
}
// the warp's sum in a fixed xor tree; lane 0's value is the one used
__device__ __forceinline__ FF ff_warp_sum(FF a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        FF b;
        b.hi = __shfl_xor_sync(0xffffffffu, a.hi, o);
        b.lo = __shfl_xor_sync(0xffffffffu, a.lo, o);
        a = ff_add(a, b);
    }
    return a;
}
__device__ __forceinline__ double ff_to_double(FF a) { return (double)a.hi + (double)a.lo; }

// ------------------------------------------------------- device structures
// Block CSR matrix with br x bc row-major blocks (nbr block rows).
struct DMat {
    int nbr = 0, nbc = 0, br = 1, bc = 1;
    int64_t nnz = 0;
    int *rp = nullptr, *ci = nullptr;
    double *v = nullptr;             // FP64 values (always present)
    float *v32 = nullptr;            // FP32 copy (mixed precision)
    __nv_bfloat16 *v16 = nullptr;    // BF16 copy (mixed precision)
    // Sliced-ELL copy for square blocks (C-row slices, C = sl_c; slot k of row
    // t of slice s at sl_ptr[s] + C k + t; its bs*bs values component-major:
    // value q of the C slots of one k at (sl_ptr[s] + C k) * bb + C q + t).
    int nslice = 0, sl_c = 32;       // number of slices, rows per slice (8 or 32)
    long long *sl_ptr = nullptr;
    int *sl_ci = nullptr;
    double *sl_v = nullptr;
    float *sl_v32 = nullptr;
    // BF16 values use a paired variant of the same slices (same widths):
    // slots 2p, 2p+1 of a row stored side by side, so that one thread loads
    // both with one 4-byte load (bf16x2) per component and one 8-byte load
    // (int2) of columns: pair slot g = sl2_ptr[s] / 2 + C p, its columns at
    // sl2_ci[2 (g + t) + h], value q at sl_v16[2 ((g bb) + C q + t) + h].  An
    // odd width w's last slot is stored unpaired after the pairs: with
    // g = sl2_ptr[s] + C (w - 1), its columns at sl2_ci[g + t], value q at
    // sl_v16[g bb + C q + t].
    long long *sl2_ptr = nullptr;
    int *sl2_ci = nullptr;
    __nv_bfloat16 *sl_v16 = nullptr;
    int tuned = -1;                  // autotuned kernel: -1 untuned, 0 sliced ELL, 1000 + T sliced ELL with T threads per row, other > 0 flat with that many lanes per row
    int bb() const { return br * bc; }
};

// Sparse rank-one data, arranged per velocity block row for the fused epilogue:
// entries lr_rp[i]..lr_rp[i+1]-1 of block row i hold (outlet k, component c, value).
struct LowRank {
    int n_out = 0;
    int no = 0;                              // entries over all outlets
    int *optr = nullptr, *oidx = nullptr;    // per-outlet sparse vectors (device)
    double *oval = nullptr;
    double *r = nullptr;                     // device copy of r_k
    std::vector<double> r_host;
    int *lr_rp = nullptr;                    // N+1
    int *lr_k = nullptr, *lr_c = nullptr;
    double *lr_val = nullptr;
    double *f = nullptr;                     // r_k (a^k . x), device, n_out
};

struct Level {
    DMat M;
    int *agg = nullptr;                      // map to next level (-1 = left out)
    int *mptr = nullptr, *mem = nullptr;     // members of each next-level aggregate
    double *dinv = nullptr;                  // bs*bs per row
    float *dinv32 = nullptr;
    double rho = 0.0;
    double cheb_lo = 10.0;                   // Chebyshev interval [rho / cheb_lo, rho]
    // work vectors: [0] b, [1] x, [2] x (ping-pong), [3] r, [4] d, and for the
    // K-cycle [5] r, [6] z1, [7] w1, [8] z2, [9] w2; FP64 and FP32 sets
    static constexpr int kWork = 10;
    double *w64[kWork] = {};
    float *w32[kWork] = {};
    double *kdots = nullptr;                 // K-cycle inner products (device)
    double *kpart = nullptr;                 // block partials of the K-cycle's product + inner products kernel
    long long kpart_blocks = 0;              // ... for grids up to this many blocks
};

struct Hier {
    int nlev = 0, bs = 1;
    bool kcycle = false;                     // Krylov-accelerated cycle on the coarse levels
    int kdepth = 1;                          // ... 1..kdepth
    int cheb = 2;                            // Chebyshev smoothing degree of this hierarchy
    Level L[kMaxLevels];
    double *cinv = nullptr;                  // coarsest dense inverse (nc x nc, row-major) or null
    float *cinv32 = nullptr;                 // its FP32 copy (FP32 inner solves)
    int nc = 0;
    bool built = false;
};

}  // namespace nbp

namespace nbp {

// ------------------------------------------------------ device memory helpers
template <typename T> inline T *dmalloc(size_t n, cudaStream_t s) {
    void *p = nullptr;
    NBP_CUDA(cudaMallocAsync(&p, (n ? n : 1) * sizeof(T), s));
    return (T *)p;
}
inline void dfree(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}
template <typename T> inline T readback(const T *d, cudaStream_t s) {
    T h;
    NBP_CUDA(cudaMemcpyAsync(&h, d, sizeof(T), cudaMemcpyDeviceToHost, s));
    NBP_CUDA(cudaStreamSynchronize(s));
    return h;
}
inline unsigned grid_for(long long n, int block = 256, long long cap = 16LL * kSMs * 8) {
    long long g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}
inline unsigned grid_exact(long long n, int block = 256) {
    long long g = (n + block - 1) / block;
    return (unsigned)(g < 1 ? 1 : g);
}

void dmat_free(DMat &m, cudaStream_t s);
void hier_free(Hier &H, cudaStream_t s);

// Setup entry points (amg_setup.cu)
// Aggregation AMG hierarchy of `fine`; keep_aggregates: rebuild every
// operator of the hierarchy H already holds (same pattern) from the new
// values on its aggregate maps instead of aggregating again.
void amg_build(Hier &H, const DMat &fine, const nbp_options &o, int precision, cudaStream_t s,
               bool keep_aggregates = false);
void build_shat(const DMat &A, const DMat &B, const DMat &C, const DMat &D, const LowRank &lr, int N, DMat &Shat,
                double *diagA_out, cudaStream_t s);
void make_lowcopies(DMat &m, int precision, cudaStream_t s);
void make_sell(DMat &m, int precision, cudaStream_t s);
void transpose_dmat(const DMat &in, DMat &out, cudaStream_t s);

}  // namespace nbp
