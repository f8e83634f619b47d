// krylov.cu -- non-template kernels of the Krylov layer: fixed-order partial
// reductions and the device Givens / least-squares update of (F)GMRES.
#include "kernels.cuh"

namespace nbp {

__global__ void k_reduce_partials(const double *__restrict__ partial, int nblocks, int ncols, double *__restrict__ out,
                                  int accumulate) {
    const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int ln = threadIdx.x & 31;
    if (col >= ncols) return;
    double s = 0.0;
    for (int b = ln; b < nblocks; b += 32) s += partial[(long long)col * nblocks + b];
    s = warp_sum(s);
    if (ln == 0) out[col] = accumulate ? out[col] + s : s;
}

// Hessenberg column j: H(i,j) = h1_i + h2_i (i <= j), H(j+1,j) = ||w||;
// previous rotations applied, new rotation chosen to zero H(j+1,j), and the
// right-hand side g rotated (Saad 1993, FGMRES with Givens rotations).
__global__ void k_givens(double *H, int ldh, int j, const double *h1, const double *h2, const double *nrm2, double *cs,
                         double *sn, double *g, GmState *st) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = 0; i <= j; ++i) H[(long long)i * ldh + j] = h1[i] + h2[i];
    const double q = nrm2[0];
    const double beta = (q >= 0.0) ? sqrt(q) : q;   // NaN passes through (fmax would hide it)
    H[(long long)(j + 1) * ldh + j] = beta;
    for (int i = 0; i < j; ++i) {
        const double a = H[(long long)i * ldh + j], b = H[(long long)(i + 1) * ldh + j];
        H[(long long)i * ldh + j] = cs[i] * a + sn[i] * b;
        H[(long long)(i + 1) * ldh + j] = -sn[i] * a + cs[i] * b;
    }
    const double a = H[(long long)j * ldh + j], b = H[(long long)(j + 1) * ldh + j];
    const double den = hypot(a, b);
    if (den == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
    else { cs[j] = a / den; sn[j] = b / den; }
    H[(long long)j * ldh + j] = den;
    H[(long long)(j + 1) * ldh + j] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    const double res = fabs(g[j + 1]);
    st->res = res;
    st->beta = beta;
    st->nan = (isfinite(res) && isfinite(beta)) ? 0 : 1;
}

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
