// spmv.cuh -- host-side dispatcher of the block-sparse product kernels.
#pragma once
#include "kernels.cuh"

namespace nbp {

// Launch y = epilogue(M x) on stream s.  vsel selects the value copy
// (0 FP64, 1 FP32, 2 BF16); XT is the vector type (double needs vsel 0).
// G = lanes per block row (0: chosen from the average row length).
template <typename XT>
void spmv(const DMat &M, int vsel, SpmvArgs a, int epi, bool lr, cudaStream_t s, int G = 0);

int choose_group(const DMat &M);

}  // namespace nbp
