// spmv.cuh -- host-side dispatcher of the block-sparse product kernels.
#pragma once
#include "kernels.cuh"

namespace nbp {

// Launch y = epilogue(M x) on stream s.  vsel selects the value copy
// (0 FP64, 1 FP32, 2 BF16); XT is the vector type (double needs vsel 0).
// G: -1 = the autotuned choice (else sliced ELL when built); 0 = sliced ELL;
// kSellMT + T = sliced ELL with T threads per row (T = 2, 4, 8); other > 0 =
// flat kernel with G lanes per block row.  Returns the product's algorithmic
// bytes (what the launched kernel must move at least: values, columns, row or
// slice pointers, x once, the epilogue's vectors), for bandwidth accounting.
template <typename XT>
double spmv(const DMat &M, int vsel, SpmvArgs a, int epi, bool lr, cudaStream_t s, int G = -1);

int choose_group(const DMat &M);

// Whether y = M x with the K-cycle's inner products fused (k_sell_dot) runs
// for this matrix: scalar blocks, the sliced kernel (1-8 threads per row) as
// the tuned choice, the value copy of vsel built, and a grid of at most
// max_blocks blocks (the partials buffer).
bool spmv_dot_ok(const DMat &M, int vsel, int xbytes, long long max_blocks);
// Launch it (spmv_dot_ok must hold); returns the algorithmic bytes: the
// product's, plus da and db when they are not y.
template <typename XT>
double spmv_dot(const DMat &M, int vsel, SpmvArgs a, const DotArgs &q, cudaStream_t s);


}  // namespace nbp
