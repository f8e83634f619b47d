// noalloc.cu -- y = A x (sparse part plus the outlet rank-one terms) without
// any device allocation, for callers that cannot call cudaMalloc: code that
// runs after a framework has frozen its memory pool, real-time or embedded
// callers that forbid allocation after start-up, and callers that hold no
// library context.  The per-outlet inner products that the regular path keeps
// in context-owned device memory live here in a fixed file-scope device array.
#include "kernels.cuh"

namespace nbp {

// Largest number of outlets one call may pass; the array costs 8 KiB of
// device memory on every GPU that loads the library, held until exit.
constexpr int kNoAllocMaxOutlets = 1024;

// Scratch shared by every call on a device: f[k] = r_k (a^k . x).  Each call
// writes all n_out entries before reading them, so nothing needs clearing;
// calls that overlap on the GPU (different streams, no ordering) race on it.
static __device__ __align__(256) double g_noalloc_f[kNoAllocMaxOutlets];

// y[idx] += f[k] * val for every outlet k in ascending order, by one block:
// the entries of one outlet have distinct indices, so its threads never touch
// the same y entry, and the barrier between outlets keeps each y entry's
// additions in ascending k (a fixed order, one launch for any n_out).
__global__ void __launch_bounds__(1024) k_noalloc_scatter(const int *__restrict__ optr, const int *__restrict__ oidx,
                                                          const double *__restrict__ oval, const double *__restrict__ f,
                                                          int n_out, double *__restrict__ y) {
    for (int k = 0; k < n_out; ++k) {
        const int beg = optr[k], end = optr[k + 1];
        const double fk = f[k];
        for (int q = beg + threadIdx.x; q < end; q += blockDim.x) y[oidx[q]] += fk * oval[q];
        __syncthreads();
    }
}

namespace {
// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// with the device current -- on every call, so that a context torn down and
// made again (a device reset) never leaves a stale address behind.  The
// lookup queues no work on any stream.
cudaError_t scratch_for_current_device(double **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_f);
    if (e != cudaSuccess) return e;
    *out = (double *)p;
    return cudaSuccess;
}
}  // namespace

}  // namespace nbp

extern "C" nbp_status nbp_apply_A_noalloc(int32_t n_nodes, const int32_t *a_rowptr, const int32_t *a_col,
                                          const double *a_val, int32_t n_out, const int32_t *out_ptr,
                                          const int32_t *out_idx, const double *out_val, const double *r,
                                          const double *x, double *y, void *stream) {
    using namespace nbp;
    if (n_nodes <= 0 || !a_rowptr || !a_col || !a_val || !x || !y) return NBP_ERR_INVALID;
    if (n_out < 0 || n_out > kNoAllocMaxOutlets) return NBP_ERR_INVALID;
    if (n_out > 0 && (!out_ptr || !out_idx || !out_val || !r)) return NBP_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    double *f = nullptr;
    if (scratch_for_current_device(&f) != cudaSuccess) return NBP_ERR_CUDA;
    if (n_out > 0) {
        k_lowrank_dots<double><<<n_out, 256, 0, s>>>(out_ptr, out_idx, out_val, r, x, f);
        if (cudaGetLastError() != cudaSuccess) return NBP_ERR_CUDA;
    }
    SpmvArgs a{};
    a.nbr = n_nodes;
    a.rp = a_rowptr;
    a.ci = a_col;
    a.val = a_val;
    a.x = x;
    a.y = y;
    const long long threads = (long long)n_nodes * 16;
    k_bspmv<3, 3, 16, double, double, EPI_SET, false><<<grid_exact(threads), 256, 0, s>>>(a);
    if (cudaGetLastError() != cudaSuccess) return NBP_ERR_CUDA;
    if (n_out > 0) {
        k_noalloc_scatter<<<1, 1024, 0, s>>>(out_ptr, out_idx, out_val, f, n_out, y);
        if (cudaGetLastError() != cudaSuccess) return NBP_ERR_CUDA;
    }
    return NBP_OK;
}
