// krylov.cu -- non-template kernels of the Krylov layer: the triangular
// solve of the GMRES least-squares problem and the start of a GMRES cycle
// (the Givens update itself is fused into the last Gram-Schmidt kernel of
// each Arnoldi step).
#include "kernels.cuh"

namespace nbp {

__device__ __forceinline__ void trisolve(const double *H, int ldh, const double *g, double *y, int k) {
    for (int i = k - 1; i >= 0; --i) {
        double s = g[i];
        for (int q = i + 1; q < k; ++q) s -= H[(long long)i * ldh + q] * y[q];
        const double d = H[(long long)i * ldh + i];
        y[i] = (d != 0.0) ? s / d : 0.0;
    }
}

__global__ void k_trisolve(const double *H, int ldh, const double *g, double *y, int k) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    trisolve(H, ldh, g, y, k);
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

// ------------------------------------------------ device-driven Krylov loops
// The loop of one GMRES level runs as a graph WHILE node; these one-thread
// (or one-block) kernels keep its state in GmDev and set the node's
// condition at the start and end of a cycle; each iteration ends in
// k_scale_step_dl, whose last block applies the stopping rule (dl_step).

__global__ void k_dl_init(GmDev *st, double *g, int m1, const double *nrm2, double *beta, GmState *gs,
                          const double *rtol, const double *atol, const int *m, const int *nmax,
                          cudaGraphConditionalHandle h) {
    for (int i = threadIdx.x; i < m1; i += blockDim.x) g[i] = 0.0;
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double q = nrm2[0];
    const double b = (q >= 0.0) ? sqrt(q) : q;   // NaN passes through
    g[0] = b;
    *beta = b;
    gs->res = b;
    gs->beta = b;
    gs->nan = isfinite(b) ? 0 : 1;
    st->j = 0;
    st->its = 0;
    st->pad0 = 0;
    st->m = *m;
    st->nmax = *nmax;
    st->bnorm = b;
    st->res = b;
    st->tol = fmax(*rtol * b, *atol);
    st->nan = isfinite(b) ? 0 : 1;
    st->conv = (b <= st->tol) ? 1 : 0;
    st->rel_true = b > 0.0 ? 1.0 : 0.0;
    cudaGraphSetConditional(h, (!st->conv && !st->nan && st->nmax > 0) ? 1u : 0u);
}

__global__ void k_dl_cycle_start(GmDev *st, cudaGraphConditionalHandle h) {
    st->j = 0;
    st->pad0 += 1;   // cycles run (counted for the kernel tally)
    cudaGraphSetConditional(h, 1u);
}

__global__ void k_dl_end(GmDev *st, const double *H, int ldh, const double *g, double *y, long long *its_total,
                         long long *solves) {
    trisolve(H, ldh, g, y, st->j);
    st->conv = st->res <= st->tol ? 1 : 0;
    if (its_total) *its_total += st->its;
    if (solves) *solves += 1;
}

__global__ void k_dl_restart(GmDev *st, const double *nrm2, double *g, int m1, double *beta, GmState *gs,
                             cudaGraphConditionalHandle h) {
    const double q = nrm2[0];
    const double r = (q >= 0.0) ? sqrt(q) : q;
    __shared__ int go;
    if (threadIdx.x == 0) {
        st->res = r;
        st->rel_true = st->bnorm > 0.0 ? r / st->bnorm : 0.0;
        if (!isfinite(r)) st->nan = 1;
        st->conv = (r <= st->tol) ? 1 : 0;
        go = (!st->conv && !st->nan && st->its < st->nmax && r != 0.0) ? 1 : 0;
    }
    __syncthreads();
    if (go) {
        for (int i = threadIdx.x; i < m1; i += blockDim.x) g[i] = 0.0;
        __syncthreads();
        if (threadIdx.x == 0) {
            g[0] = r;
            *beta = r;
            gs->res = r;
            gs->beta = r;
            gs->nan = 0;
        }
    }
    if (threadIdx.x == 0) cudaGraphSetConditional(h, go ? 1u : 0u);
}

}  // namespace nbp
