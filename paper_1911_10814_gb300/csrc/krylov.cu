// krylov.cu -- non-template kernels of the Krylov layer: the triangular
// solve of the GMRES least-squares problem and the start of a GMRES cycle
// (the Givens update itself is fused into the last Gram-Schmidt kernel of
// each Arnoldi step).
#include "kernels.cuh"

namespace nbp {

__global__ void k_trisolve(const double *H, int ldh, const double *g, double *y, int k) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = k - 1; i >= 0; --i) {
        double s = g[i];
        for (int q = i + 1; q < k; ++q) s -= H[(long long)i * ldh + q] * y[q];
        const double d = H[(long long)i * ldh + i];
        y[i] = (d != 0.0) ? s / d : 0.0;
    }
}

__global__ void k_gm_init(double *g, int m1, const double *beta2, double *beta, GmState *st) {
    const double q = beta2[0];
    const double b = (q >= 0.0) ? sqrt(q) : q;       // NaN passes through (fmax would hide it)
    for (int i = threadIdx.x; i < m1; i += blockDim.x) g[i] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
        g[0] = b;
        *beta = b;
        st->res = b;
        st->beta = b;
        st->nan = isfinite(b) ? 0 : 1;
    }
}

}  // namespace nbp
