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


}  // namespace nbp
