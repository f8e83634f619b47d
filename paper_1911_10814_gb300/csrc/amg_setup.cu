// amg_setup.cu -- on-device setup of the nested block solver: aggregation AMG
// hierarchies (strength, handshake matching, aggregate numbering, Galerkin
// product, block-diagonal inverses, Gershgorin bounds, dense coarsest
// inverse), the sparse Schur approximation S_hat = D - C diag(A)^{-1} B
// (paper Sec. 3.1), value copies for mixed precision, and block transposes
// for the adjoint.
//
// Aggregation rule (the paper uses BoomerAMG, Table 1, as prior art; this
// rule is the project's, and the integer aggregate maps are reproducible
// bit for bit because every decision is taken on values computed with the
// same IEEE operations in the same order, with no fused multiply-add):
//   sigma_ij = 0.5 (|A_ij|_F^2 + |A_ji|_F^2) / sqrt(|A_ii|_F^2 |A_jj|_F^2),
//   strong iff sigma_ij >= theta; 3 passes of 64 synchronous handshake rounds
//   (strongest unmatched strong neighbour, ties to the smaller index), pass
//   k+1 on the aggregate graph with max-reduced weights; aggregates numbered
//   by smallest fine index; nodes without any strong connection left out.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "kernels.cuh"

namespace nbp {

constexpr int kMatchRounds = 64;   // rounds per matching pass (extra rounds after convergence are no-ops)

// ------------------------------------------------------------- utilities
void dmat_free(DMat &m, cudaStream_t s) {
    dfree(m.rp, s); dfree(m.ci, s); dfree(m.v, s); dfree(m.v32, s); dfree(m.v16, s);
    dfree(m.sl_ptr, s); dfree(m.sl_ci, s); dfree(m.sl_v, s); dfree(m.sl_v32, s); dfree(m.sl_v16, s);
    dfree(m.sl2_ptr, s); dfree(m.sl2_ci, s);
    m = DMat();
}

void hier_free(Hier &H, cudaStream_t s) {
    for (int l = 0; l < H.nlev; ++l) {
        Level &L = H.L[l];
        dmat_free(L.M, s);
        dfree(L.agg, s); dfree(L.mptr, s); dfree(L.mem, s); dfree(L.dinv, s); dfree(L.dinv32, s);
        for (int q = 0; q < Level::kWork; ++q) { dfree(L.w64[q], s); dfree(L.w32[q], s); }
        dfree(L.kdots, s); dfree(L.kpart, s);
        L = Level();
    }
    dfree(H.cinv, s);
    dfree(H.cinv32, s);
    H = Hier();
}

template <typename T> static void exclusive_scan(const T *in, T *out, long long n, cudaStream_t s) {
    size_t bytes = 0;
    NBP_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, bytes, in, out, (int)n, s));
    void *tmp = dmalloc<char>(bytes, s);
    NBP_CUDA(cub::DeviceScan::ExclusiveSum(tmp, bytes, in, out, (int)n, s));
    dfree(tmp, s);
}

template <typename K, typename V>
static void sort_pairs(K *&keys, V *&vals, long long n, int end_bit, cudaStream_t s) {
    require(n < (1LL << 31), NBP_ERR_INVALID, "setup: sort of more than 2^31 items");
    K *k2 = dmalloc<K>(n, s);
    V *v2 = dmalloc<V>(n, s);
    size_t bytes = 0;
    NBP_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, bytes, keys, k2, vals, v2, (int)n, 0, end_bit, s));
    void *tmp = dmalloc<char>(bytes, s);
    NBP_CUDA(cub::DeviceRadixSort::SortPairs(tmp, bytes, keys, k2, vals, v2, (int)n, 0, end_bit, s));
    dfree(tmp, s);
    dfree(keys, s); dfree(vals, s);
    keys = k2; vals = v2;
}

static int bits_for(unsigned long long maxkey) {
    int b = 1;
    while (b < 64 && (maxkey >> b) != 0ULL) ++b;
    return b;
}

__device__ __forceinline__ double fnorm2_rn(const double *blk, int nb) {
    double s = __dmul_rn(blk[0], blk[0]);
    for (int t = 1; t < nb; ++t) s = __dadd_rn(s, __dmul_rn(blk[t], blk[t]));
    return s;
}

__device__ __forceinline__ int find_entry(const int *rp, const int *ci, int i, int j) {
    int lo = rp[i], hi = rp[i + 1] - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int c = ci[mid];
        if (c == j) return mid;
        if (c < j) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

// ------------------------------------------------------ strength graph
__global__ void k_diag_norm(int n, int nb, const int *rp, const int *ci, const double *v, double *dn) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int e = find_entry(rp, ci, i, i);
    dn[i] = (e >= 0) ? fnorm2_rn(v + (long long)e * nb, nb) : 0.0;
}

// w[e] = sigma_ij for off-diagonal entries, -1 on the diagonal
__global__ void k_strength(int n, int nb, const int *rp, const int *ci, const double *v, const double *dn, double *w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
        const int j = ci[e];
        if (j == i) { w[e] = -1.0; continue; }
        const double fij = fnorm2_rn(v + (long long)e * nb, nb);
        const int et = find_entry(rp, ci, j, i);
        const double fji = (et >= 0) ? fnorm2_rn(v + (long long)et * nb, nb) : 0.0;
        const double d = __dmul_rn(dn[i], dn[j]);
        const double h = __dmul_rn(__dadd_rn(fij, fji), 0.5);
        w[e] = (d > 0.0) ? __ddiv_rn(h, __dsqrt_rn(d)) : 0.0;
    }
}

__global__ void k_isolated(int n, const int *rp, const int *ci, const double *w, double theta, int *iso) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int is = 1;
    for (int e = rp[i]; e < rp[i + 1]; ++e)
        if (ci[e] != i && w[e] >= theta) { is = 0; break; }
    iso[i] = is;
}

// --------------------------------------------------------- matching pass
__global__ void k_pick(int n, const int *rp, const int *ci, const double *w, double theta, const int *mate, int *pick) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    int p = -1;
    if (mate[u] < 0) {
        double best = 0.0;
        for (int e = rp[u]; e < rp[u + 1]; ++e) {
            const int v = ci[e];
            if (v == u || mate[v] >= 0) continue;
            const double wv = w[e];
            if (!(wv >= theta)) continue;
            if (p < 0 || wv > best || (wv == best && v < p)) { best = wv; p = v; }
        }
    }
    pick[u] = p;
}

__global__ void k_match(int n, const int *pick, int *mate) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    const int v = pick[u];
    if (v >= 0 && pick[v] == u) mate[u] = v;
}

__global__ void k_root_flag(int n, const int *mate, int *flag) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    const int m = mate[u];
    flag[u] = (m < 0 || m > u) ? 1 : 0;
}

__global__ void k_map_from_roots(int n, const int *mate, const int *id, int *map) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    const int m = mate[u];
    map[u] = (m >= 0 && m < u) ? id[m] : id[u];
}

__global__ void k_compose(int n, const int *map, int *agg) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    agg[i] = map[agg[i]];
}

__global__ void k_iota(int n, int *a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = i;
}

// row index of every stored entry
__global__ void k_entry_rows(int n, const int *rp, int *row) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int e = rp[i]; e < rp[i + 1]; ++e) row[e] = i;
}

// keys of an aggregate graph: (map[u], map[v]) for u != v aggregates, sentinel otherwise
__global__ void k_cg_keys(long long nnz, const int *row, const int *ci, const int *map, unsigned long long ncl,
                          int drop_diag, unsigned long long *key, long long *idx) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    const int I = map[row[e]], J = map[ci[e]];
    const bool drop = I < 0 || J < 0 || (drop_diag && I == J);
    key[e] = drop ? ~0ULL : (unsigned long long)I * ncl + (unsigned long long)J;
    idx[e] = e;
}

// segment heads of sorted keys (sentinel keys are never heads)
__global__ void k_heads(long long n, const unsigned long long *key, int *head) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const unsigned long long k = key[t];
    head[t] = (k != ~0ULL && (t == 0 || key[t - 1] != k)) ? 1 : 0;
}

// start position of each segment; segment s = sid[t] for heads
__global__ void k_seg_starts(long long n, const int *head, const int *sid, long long *start) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    if (head[t]) start[sid[t]] = t;
}

// coarse graph rows: count per row then scan
__global__ void k_seg_rowcount(int nseg, const unsigned long long *key, const long long *start, unsigned long long ncl,
                               int *cnt) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    const unsigned long long k = key[start[s]];
    atomicAdd(cnt + (int)(k / ncl), 1);
}

// aggregate graph edges: column and max weight over the segment
__global__ void k_cg_fill(int nseg, const unsigned long long *key, const long long *start, long long nvalid,
                          const long long *idx, const double *w, unsigned long long ncl, int *ci_out, double *w_out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    const long long a = start[s];
    const long long b = (s + 1 < nseg) ? start[s + 1] : nvalid;
    const unsigned long long k = key[a];
    double m = w[idx[a]];
    for (long long t = a + 1; t < b; ++t) m = fmax(m, w[idx[t]]);
    ci_out[s] = (int)(k % ncl);
    w_out[s] = m;
}

// Galerkin: coarse block = sequential sum of the segment's fine blocks in
// ascending fine entry order (ascending (row, column))
__global__ void k_galerkin_fill(int nseg, int nb, const unsigned long long *key, const long long *start, long long nvalid,
                                const long long *idx, const double *v, unsigned long long ncl, int *ci_out, double *v_out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    const long long a = start[s];
    const long long b = (s + 1 < nseg) ? start[s + 1] : nvalid;
    ci_out[s] = (int)(key[a] % ncl);
    double acc[9];
    const double *src = v + idx[a] * nb;
    for (int q = 0; q < nb; ++q) acc[q] = src[q];
    for (long long t = a + 1; t < b; ++t) {
        src = v + idx[t] * nb;
        for (int q = 0; q < nb; ++q) acc[q] = __dadd_rn(acc[q], src[q]);
    }
    for (int q = 0; q < nb; ++q) v_out[(long long)s * nb + q] = acc[q];
}

__global__ void k_count_valid(long long n, const unsigned long long *key, unsigned long long *cnt) {
    // number of non-sentinel keys = position of the first sentinel (keys sorted)
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const bool valid = key[t] != ~0ULL;
    const bool next_invalid = (t + 1 == n) || key[t + 1] == ~0ULL;
    if (valid && next_invalid) *cnt = (unsigned long long)(t + 1);
}

// keep flags of aggregates holding at least one non-isolated node
__global__ void k_mark_keep(int n, const int *agg, const int *iso, int *keep) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (!iso[i]) keep[agg[i]] = 1;
}
__global__ void k_drop_isolated(int n, const int *iso, const int *newid, int *agg) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    agg[i] = iso[i] ? -1 : newid[agg[i]];
}

// ---------------------------------------------------- diagonal inverses
__global__ void k_block_dinv(int n, int bs, const int *rp, const int *ci, const double *v, double *dinv, int *singular) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int e = find_entry(rp, ci, i, i);
    double *o = dinv + (long long)i * bs * bs;
    if (bs == 1) {
        const double a = (e >= 0) ? v[e] : 0.0;
        o[0] = (a != 0.0) ? 1.0 / a : 0.0;
        if (a == 0.0) atomicAdd(singular, 1);
        return;
    }
    double a[9];
    for (int q = 0; q < 9; ++q) a[q] = (e >= 0) ? v[(long long)e * 9 + q] : 0.0;
    const double c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8], c02 = a[3] * a[7] - a[4] * a[6];
    const double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
    if (det == 0.0) {
        for (int q = 0; q < 9; ++q) o[q] = 0.0;
        atomicAdd(singular, 1);
        return;
    }
    const double id = 1.0 / det;
    o[0] = c00 * id; o[1] = (a[2] * a[7] - a[1] * a[8]) * id; o[2] = (a[1] * a[5] - a[2] * a[4]) * id;
    o[3] = c01 * id; o[4] = (a[0] * a[8] - a[2] * a[6]) * id; o[5] = (a[2] * a[3] - a[0] * a[5]) * id;
    o[6] = c02 * id; o[7] = (a[1] * a[6] - a[0] * a[7]) * id; o[8] = (a[0] * a[4] - a[1] * a[3]) * id;
}

// Gershgorin bound of D_b^{-1} A: max over scalar rows of sum |(D_b^{-1} A)_rc|
__global__ void k_gershgorin(int n, int bs, const int *rp, const double *v, const double *dinv, unsigned long long *rho_bits) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int nb = bs * bs;
    const double *di = dinv + (long long)i * nb;
    double mx = 0.0;
    for (int a = 0; a < bs; ++a) {
        double s = 0.0;
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            const double *blk = v + (long long)e * nb;
            for (int c = 0; c < bs; ++c) {
                double t = 0.0;
                for (int k = 0; k < bs; ++k) t += di[a * bs + k] * blk[k * bs + c];
                s += fabs(t);
            }
        }
        mx = fmax(mx, s);
    }
    atomicMax(rho_bits, (unsigned long long)__double_as_longlong(mx));   // order-free for x >= 0
}

// --------------------------------------------------- dense coarsest solve
__global__ void k_dense_from_bsr(int nbr, int bs, const int *rp, const int *ci, const double *v, double *Dm) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nbr) return;
    const int n = nbr * bs, nb = bs * bs;
    for (int e = rp[i]; e < rp[i + 1]; ++e)
        for (int a = 0; a < bs; ++a)
            for (int b = 0; b < bs; ++b)
                Dm[(long long)(i * bs + a) * n + (long long)ci[e] * bs + b] += v[(long long)e * nb + a * bs + b];
}
__global__ void k_identity(int n, double *I) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * n) return;
    I[t] = ((t / n) == (t % n)) ? 1.0 : 0.0;
}
// Gauss-Jordan step k with partial pivoting on [M | Inv] (one block)
__global__ void k_gj_pivot(int n, int k, double *M, double *Inv, int *fail) {
    __shared__ double bv[1024];
    __shared__ int bi[1024];
    double best = -1.0;
    int arg = k;
    for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
        const double a = fabs(M[(long long)i * n + k]);
        if (a > best || (a == best && i < arg)) { best = a; arg = i; }
    }
    bv[threadIdx.x] = best; bi[threadIdx.x] = arg;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            const double o = bv[threadIdx.x + s];
            const int oi = bi[threadIdx.x + s];
            if (o > bv[threadIdx.x] || (o == bv[threadIdx.x] && oi < bi[threadIdx.x])) { bv[threadIdx.x] = o; bi[threadIdx.x] = oi; }
        }
        __syncthreads();
    }
    const int p = bi[0];
    const double piv = M[(long long)p * n + k];
    if (piv == 0.0) { if (threadIdx.x == 0) *fail = 1; return; }
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        if (p != k) {
            double t = M[(long long)k * n + c]; M[(long long)k * n + c] = M[(long long)p * n + c]; M[(long long)p * n + c] = t;
            t = Inv[(long long)k * n + c]; Inv[(long long)k * n + c] = Inv[(long long)p * n + c]; Inv[(long long)p * n + c] = t;
        }
    }
    __syncthreads();
    const double ip = 1.0 / piv;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        M[(long long)k * n + c] *= ip;
        Inv[(long long)k * n + c] *= ip;
    }
}
__global__ void k_gj_elim(int n, int k, double *M, double *Inv, const int *fail) {
    if (*fail) return;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * 2 * n) return;
    const int i = (int)(t / (2 * n));
    const int c = (int)(t % (2 * n));
    if (i == k) return;
    const double f = M[(long long)i * n + k];
    if (c < n) {
        if (c == k) return;   // column k cleared last (it is the factor)
        M[(long long)i * n + c] -= f * M[(long long)k * n + c];
    } else {
        Inv[(long long)i * n + (c - n)] -= f * Inv[(long long)k * n + (c - n)];
    }
}
__global__ void k_gj_clear(int n, int k, double *M) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || i == k) return;
    M[(long long)i * n + k] = 0.0;
}

// --------------------------------------------------- value copies
__global__ void k_to_f32(const double *a, float *b, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) b[i] = (float)a[i];
}
__global__ void k_to_bf16(const double *a, __nv_bfloat16 *b, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = __float2bfloat16_rn((float)a[i]);
}

// ------------------------------------------------------------ sliced ELL
__global__ void k_sell_width(int nbr, int nslice, int C, const int *rp, long long *slots) {
    const int sl = blockIdx.x * blockDim.x + threadIdx.x;
    if (sl >= nslice) return;
    int w = 0;
    for (int t = 0; t < C; ++t) {
        const int i = sl * C + t;
        if (i < nbr) w = max(w, rp[i + 1] - rp[i]);
    }
    slots[sl] = (long long)C * w;
}
// BF16 values and columns in the paired layout (see DMat::sl2_ptr)
__global__ void k_sell_fill2(int nbr, int nslice, int C, int bb, const int *rp, const int *ci, const double *v,
                             const long long *sp2, int *sci2, __nv_bfloat16 *sv16) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int sl = row / C, t = row % C;
    if (sl >= nslice) return;
    const long long base = sp2[sl], base2 = base / 2;
    const int w = (int)((sp2[sl + 1] - base) / C);
    const int len = (row < nbr) ? rp[row + 1] - rp[row] : 0;
    const int e0 = (row < nbr) ? rp[row] : 0;
    for (int k = 0; k < w; ++k) {
        const bool real = k < len;
        const int col = real ? ci[e0 + k] : 0;
        if (k < (w & ~1)) {   // slot of pair k / 2
            const long long g = base2 + (long long)C * (k >> 1);
            const int h = k & 1;
            sci2[2 * (g + t) + h] = col;
            for (int q = 0; q < bb; ++q) {
                const double val = real ? v[(long long)(e0 + k) * bb + q] : 0.0;
                sv16[2 * (g * bb + (long long)C * q + t) + h] = __float2bfloat16_rn((float)val);
            }
        } else {              // the unpaired last slot of an odd width
            const long long g = base + (long long)C * k;
            sci2[g + t] = col;
            for (int q = 0; q < bb; ++q) {
                const double val = real ? v[(long long)(e0 + k) * bb + q] : 0.0;
                sv16[g * bb + (long long)C * q + t] = __float2bfloat16_rn((float)val);
            }
        }
    }
}
__global__ void k_sell_fill(int nbr, int nslice, int C, int bb, const int *rp, const int *ci, const double *v,
                            const long long *sp, int *sci, double *sv, float *sv32) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int sl = row / C, t = row % C;
    if (sl >= nslice) return;
    const long long base = sp[sl];
    const int w = (int)((sp[sl + 1] - base) / C);
    const int len = (row < nbr) ? rp[row + 1] - rp[row] : 0;
    const int e0 = (row < nbr) ? rp[row] : 0;
    for (int k = 0; k < w; ++k) {
        const long long g = base + (long long)C * k;
        const bool real = k < len;
        sci[g + t] = real ? ci[e0 + k] : 0;
        for (int q = 0; q < bb; ++q) {
            const double val = real ? v[(long long)(e0 + k) * bb + q] : 0.0;
            const long long o = g * bb + (long long)C * q + t;
            sv[o] = val;
            if (sv32) sv32[o] = (float)val;
        }
    }
}

// slice pointers for slice height C; returns the padded slot count
static long long sell_layout(const DMat &m, int C, long long *&sp, cudaStream_t s) {
    const int ns = (m.nbr + C - 1) / C;
    long long *slots = dmalloc<long long>(ns + 1, s);
    k_sell_width<<<grid_exact(ns), 256, 0, s>>>(m.nbr, ns, C, m.rp, slots);
    NBP_LAUNCHED();
    NBP_CUDA(cudaMemsetAsync(slots + ns, 0, sizeof(long long), s));
    sp = dmalloc<long long>(ns + 1, s);
    exclusive_scan(slots, sp, ns + 1, s);
    dfree(slots, s);
    return readback(sp + ns, s);
}

// Slice layout: 32-row slices unless their padding exceeds 10 % of the
// stored blocks, else 8-row slices.  The paired BF16 layout uses the same
// slices: every slot is stored, an odd width's last slot unpaired.  (Rows
// sorted by length within windows of 256 rows cut the padding of the coarse
// levels by 15-30 % but made their products slower: the rows that a warp
// takes no longer share their neighbours' x entries.)
void make_sell(DMat &m, int precision, cudaStream_t s) {
    if (m.nbr == 0) return;
    if (m.sl_ci && (precision < 1 || m.sl_v32) && (precision < 2 || m.sl_v16)) return;   // 2, 3: FP32 and BF16
    dfree(m.sl_ptr, s); dfree(m.sl_ci, s); dfree(m.sl_v, s); dfree(m.sl_v32, s); dfree(m.sl_v16, s);
    dfree(m.sl2_ptr, s); dfree(m.sl2_ci, s);
    m.sl_ptr = nullptr; m.sl_ci = nullptr; m.sl_v = nullptr; m.sl_v32 = nullptr; m.sl_v16 = nullptr;
    m.sl2_ptr = nullptr; m.sl2_ci = nullptr;
    int C = 32;
    long long total = sell_layout(m, 32, m.sl_ptr, s);
    if (total > m.nnz + m.nnz / 10) {
        dfree(m.sl_ptr, s);
        C = 8;
        total = sell_layout(m, 8, m.sl_ptr, s);
    }
    m.sl_c = C;
    m.nslice = (m.nbr + C - 1) / C;
    const int bb = m.bb();
    m.sl_ci = dmalloc<int>(total, s);
    m.sl_v = dmalloc<double>(total * bb, s);
    if (precision >= 1) m.sl_v32 = dmalloc<float>(total * bb, s);
    k_sell_fill<<<grid_exact((long long)m.nslice * C), 256, 0, s>>>(m.nbr, m.nslice, C, bb, m.rp, m.ci, m.v, m.sl_ptr,
                                                                    m.sl_ci, m.sl_v, m.sl_v32);
    NBP_LAUNCHED();
    if (precision >= 2) {   // BF16: paired layout over the same slices
        m.sl2_ptr = dmalloc<long long>(m.nslice + 1, s);
        NBP_CUDA(cudaMemcpyAsync(m.sl2_ptr, m.sl_ptr, sizeof(long long) * (m.nslice + 1), cudaMemcpyDeviceToDevice, s));
        m.sl2_ci = dmalloc<int>(total, s);
        m.sl_v16 = dmalloc<__nv_bfloat16>(total * bb, s);
        k_sell_fill2<<<grid_exact((long long)m.nslice * C), 256, 0, s>>>(m.nbr, m.nslice, C, bb, m.rp, m.ci, m.v,
                                                                         m.sl2_ptr, m.sl2_ci, m.sl_v16);
        NBP_LAUNCHED();
    }
}

void make_lowcopies(DMat &m, int precision, cudaStream_t s) {
    const long long nv = m.nnz * m.bb();
    if (precision >= 1 && !m.v32) {
        m.v32 = dmalloc<float>(nv, s);
        k_to_f32<<<grid_for(nv), 256, 0, s>>>(m.v, m.v32, nv);
        NBP_LAUNCHED();
    }
    if (precision >= 2 && !m.v16) {
        m.v16 = dmalloc<__nv_bfloat16>(nv, s);
        k_to_bf16<<<grid_for(nv), 256, 0, s>>>(m.v, m.v16, nv);
        NBP_LAUNCHED();
    }
}

// ================================================================ aggregation
struct Graph {
    int n = 0;
    long long nnz = 0;
    int *rp = nullptr, *ci = nullptr;
    double *w = nullptr;
};
static void graph_free(Graph &g, cudaStream_t s) { dfree(g.rp, s); dfree(g.ci, s); dfree(g.w, s); g = Graph(); }

// Sort entries by (map[row], map[col]) and return segments.
struct Segments {
    unsigned long long *key = nullptr;
    long long *idx = nullptr;
    long long *start = nullptr;
    long long nvalid = 0;
    int nseg = 0;
};
static void free_segments(Segments &sg, cudaStream_t s) { dfree(sg.key, s); dfree(sg.idx, s); dfree(sg.start, s); sg = Segments(); }

static Segments group_by_coarse(int n, long long nnz, const int *rp, const int *ci, const int *map, int ncl, int drop_diag,
                                cudaStream_t s) {
    Segments sg;
    if (nnz == 0 || ncl == 0) return sg;
    int *row = dmalloc<int>(nnz, s);
    k_entry_rows<<<grid_exact(n), 256, 0, s>>>(n, rp, row);
    NBP_LAUNCHED();
    sg.key = dmalloc<unsigned long long>(nnz, s);
    sg.idx = dmalloc<long long>(nnz, s);
    k_cg_keys<<<grid_exact(nnz), 256, 0, s>>>(nnz, row, ci, map, (unsigned long long)ncl, drop_diag, sg.key, sg.idx);
    NBP_LAUNCHED();
    dfree(row, s);
    // full 64-bit sort so that the sentinel (all ones) lands last
    sort_pairs(sg.key, sg.idx, nnz, 64, s);
    unsigned long long *cnt = dmalloc<unsigned long long>(1, s);
    NBP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
    k_count_valid<<<grid_exact(nnz), 256, 0, s>>>(nnz, sg.key, cnt);
    NBP_LAUNCHED();
    sg.nvalid = (long long)readback(cnt, s);
    dfree(cnt, s);
    if (sg.nvalid == 0) return sg;
    int *head = dmalloc<int>(sg.nvalid + 1, s), *sid = dmalloc<int>(sg.nvalid + 1, s);
    k_heads<<<grid_exact(sg.nvalid), 256, 0, s>>>(sg.nvalid, sg.key, head);
    NBP_LAUNCHED();
    NBP_CUDA(cudaMemsetAsync(head + sg.nvalid, 0, sizeof(int), s));
    exclusive_scan(head, sid, sg.nvalid + 1, s);
    sg.nseg = readback(sid + sg.nvalid, s);
    sg.start = dmalloc<long long>(sg.nseg + 1, s);
    k_seg_starts<<<grid_exact(sg.nvalid), 256, 0, s>>>(sg.nvalid, head, sid, sg.start);
    NBP_LAUNCHED();
    dfree(head, s); dfree(sid, s);
    return sg;
}

static int *rowptr_from_segments(const Segments &sg, int ncl, cudaStream_t s) {
    int *cnt = dmalloc<int>(ncl + 1, s);
    NBP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (ncl + 1), s));
    if (sg.nseg > 0) {
        k_seg_rowcount<<<grid_exact(sg.nseg), 256, 0, s>>>(sg.nseg, sg.key, sg.start, (unsigned long long)ncl, cnt);
        NBP_LAUNCHED();
    }
    int *rp = dmalloc<int>(ncl + 1, s);
    exclusive_scan(cnt, rp, ncl + 1, s);
    dfree(cnt, s);
    return rp;
}

// One matching pass on G; map (n) gets aggregate ids; returns the count.
static int match_pass(const Graph &G, double theta, int *map, cudaStream_t s) {
    const int n = G.n;
    int *mate = dmalloc<int>(n, s), *pick = dmalloc<int>(n, s);
    k_fill<int><<<grid_for(n), 256, 0, s>>>(mate, -1, n);
    NBP_LAUNCHED();
    for (int round = 0; round < kMatchRounds; ++round) {   // a round without a new pair changes nothing after it
        k_pick<<<grid_exact(n), 256, 0, s>>>(n, G.rp, G.ci, G.w, theta, mate, pick);
        k_match<<<grid_exact(n), 256, 0, s>>>(n, pick, mate);
        NBP_LAUNCHED();
    }
    int *flag = dmalloc<int>(n + 1, s), *id = dmalloc<int>(n + 1, s);
    k_root_flag<<<grid_exact(n), 256, 0, s>>>(n, mate, flag);
    NBP_LAUNCHED();
    NBP_CUDA(cudaMemsetAsync(flag + n, 0, sizeof(int), s));
    exclusive_scan(flag, id, n + 1, s);
    const int nc = readback(id + n, s);
    k_map_from_roots<<<grid_exact(n), 256, 0, s>>>(n, mate, id, map);
    NBP_LAUNCHED();
    dfree(mate, s); dfree(pick, s); dfree(flag, s); dfree(id, s);
    return nc;
}

// ---- coarse rows one per warp: coarse row I gathers its members' entries
// (members ascending, each row's entries in order: ascending fine entry
// index q), maps their columns (dropping map < 0 and, for the graph, I
// itself), sorts them in shared memory by (coarse column, q), and reduces
// each coarse column's entries in order q -- the order of the global sort's
// segments, so the results are the same bit for bit.  For coarse rows of at
// most kGroupCap entries.
constexpr int kGroupCap = 1024;
constexpr int kGroupWarps = 4;   // warps per block (shared: 8 bytes per entry)

// Entries of coarse row I into sk (key = J * kGroupCap + q, padded with ~0u
// to the sort length L, the power of two >= 32 at or above the entry count)
// and their fine entry index into se[q]; returns L, and the number of
// entries kept (dropped ones sort last) in *kept.
__device__ __forceinline__ int group_row_entries(int I, int lane, const int *mptr, const int *mem, const int *rp,
                                                 const int *ci, const int *map, int drop_diag, unsigned *sk, int *se,
                                                 int *kept) {
    const int m0 = mptr[I], nm = mptr[I + 1] - m0;
    int off = 0;
    for (int a0 = 0; a0 < nm; a0 += 32) {   // members, a lane each; their entries at off + prefix
        const int a = a0 + lane;
        const int i = a < nm ? mem[m0 + a] : 0;
        const int len = a < nm ? rp[i + 1] - rp[i] : 0;
        int incl = len;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int start = off + incl - len;
        for (int f = 0; f < len; ++f) {
            const int e = rp[i] + f, q = start + f;
            const int J = map[ci[e]];
            const bool keep = J >= 0 && !(drop_diag && J == I);
            sk[q] = keep ? (((unsigned)J * (unsigned)kGroupCap) | (unsigned)q) : ~0u;
            se[q] = e;
        }
        off += __shfl_sync(0xffffffffu, incl, 31);
    }
    int L = 32;
    while (L < off) L <<= 1;
    for (int q = off + lane; q < L; q += 32) sk[q] = ~0u;
    __syncwarp();
    for (int k = 2; k <= L; k <<= 1) {   // bitonic sort, ascending
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int p = lane; p < L; p += 32) {
                const int x = p ^ j;
                if (x > p) {
                    const unsigned u = sk[p], w = sk[x];
                    if ((u > w) == ((p & k) == 0)) { sk[p] = w; sk[x] = u; }
                }
            }
            __syncwarp();
        }
    }
    int c = 0;
    for (int p = lane; p < off; p += 32) c += sk[p] != ~0u ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    *kept = c;
    return L;
}

__global__ void __launch_bounds__(32 * kGroupWarps) k_group_count(int nc, const int *mptr, const int *mem, const int *rp,
                                                                 const int *ci, const int *map, int drop_diag, int *cnt) {
    __shared__ unsigned keys[kGroupWarps][kGroupCap];
    __shared__ int ents[kGroupWarps][kGroupCap];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int I = blockIdx.x * kGroupWarps + w;
    if (I >= nc) return;
    unsigned *sk = keys[w];
    int n;
    group_row_entries(I, lane, mptr, mem, rp, ci, map, drop_diag, sk, ents[w], &n);
    int c = 0;
    for (int p = lane; p < n; p += 32) c += (p == 0 || sk[p] / kGroupCap != sk[p - 1] / kGroupCap) ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) cnt[I] = c;
}

// MAX: the graph's edge weight, fmax over the coarse column's entries (one
// value per entry); otherwise the Galerkin block, the sum of nb values per
// entry in order q
template <bool MAX>
__global__ void __launch_bounds__(32 * kGroupWarps) k_group_fill(int nc, const int *mptr, const int *mem, const int *rp,
                                                                const int *ci, const int *map, int drop_diag, int nb,
                                                                const double *v, const int *rp_out, int *ci_out,
                                                                double *v_out) {
    __shared__ unsigned keys[kGroupWarps][kGroupCap];
    __shared__ int ents[kGroupWarps][kGroupCap];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int I = blockIdx.x * kGroupWarps + w;
    if (I >= nc) return;
    unsigned *sk = keys[w];
    const int *se = ents[w];
    int n;
    const int P = group_row_entries(I, lane, mptr, mem, rp, ci, map, drop_diag, sk, ents[w], &n) / 32;
    const int p0 = lane * P;   // P contiguous positions per lane
    int mine = 0;
    for (int u = 0; u < P; ++u) {
        const int p = p0 + u;
        mine += (p < n && (p == 0 || sk[p] / kGroupCap != sk[p - 1] / kGroupCap)) ? 1 : 0;
    }
    int incl = mine;
    for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += x;
    }
    long long slot = (long long)rp_out[I] + incl - mine;
    for (int u = 0; u < P; ++u) {
        const int p = p0 + u;
        if (!(p < n && (p == 0 || sk[p] / kGroupCap != sk[p - 1] / kGroupCap))) continue;
        const unsigned J = sk[p] / kGroupCap;
        ci_out[slot] = (int)J;
        if (MAX) {
            double m = v[se[sk[p] % kGroupCap]];
            for (int r = p + 1; r < n && sk[r] / kGroupCap == J; ++r) m = fmax(m, v[se[sk[r] % kGroupCap]]);
            v_out[slot] = m;
        } else {
            double acc[9];
            const double *src = v + (long long)se[sk[p] % kGroupCap] * nb;
            for (int q = 0; q < nb; ++q) acc[q] = src[q];
            for (int r = p + 1; r < n && sk[r] / kGroupCap == J; ++r) {
                src = v + (long long)se[sk[r] % kGroupCap] * nb;
                for (int q = 0; q < nb; ++q) acc[q] = __dadd_rn(acc[q], src[q]);
            }
            for (int q = 0; q < nb; ++q) v_out[slot * nb + q] = acc[q];
        }
        ++slot;
    }
}

// entries of each coarse row before any drop (members' row lengths summed)
__global__ void k_group_size(int nc, const int *mptr, const int *mem, const int *rp, unsigned long long *mx) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    long long t = 0;
    for (int a = mptr[I]; a < mptr[I + 1]; ++a) t += rp[mem[a] + 1] - rp[mem[a]];
    atomicMax(mx, (unsigned long long)t);
}

// Coarse CSR (rp, ci, values) from the per-row grouping; false, with nothing
// made, when a coarse row holds more than kGroupCap entries or the columns
// would not fit the keys
template <bool MAX>
static bool group_rows_local(int nc, const int *mptr, const int *mem, const int *rp, const int *ci, const int *map,
                             int drop_diag, int nb, const double *v, int *&rp_out, int *&ci_out, double *&v_out,
                             long long &nnz_out, cudaStream_t s) {
    if (nc <= 0 || (unsigned long long)nc * kGroupCap >= (1ULL << 32)) return false;
    unsigned long long *mx = dmalloc<unsigned long long>(1, s);
    NBP_CUDA(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), s));
    k_group_size<<<grid_exact(nc), 256, 0, s>>>(nc, mptr, mem, rp, mx);
    NBP_LAUNCHED();
    const unsigned long long most = readback(mx, s);
    dfree(mx, s);
    if (most > (unsigned long long)kGroupCap) return false;
    const unsigned blocks = (unsigned)((nc + kGroupWarps - 1) / kGroupWarps);
    int *cnt = dmalloc<int>(nc + 1, s);
    k_group_count<<<blocks, 32 * kGroupWarps, 0, s>>>(nc, mptr, mem, rp, ci, map, drop_diag, cnt);
    NBP_LAUNCHED();
    NBP_CUDA(cudaMemsetAsync(cnt + nc, 0, sizeof(int), s));
    rp_out = dmalloc<int>(nc + 1, s);
    exclusive_scan(cnt, rp_out, nc + 1, s);
    dfree(cnt, s);
    nnz_out = readback(rp_out + nc, s);
    ci_out = dmalloc<int>(nnz_out > 0 ? nnz_out : 1, s);
    v_out = dmalloc<double>((nnz_out > 0 ? nnz_out : 1) * nb, s);
    k_group_fill<MAX><<<blocks, 32 * kGroupWarps, 0, s>>>(nc, mptr, mem, rp, ci, map, drop_diag, nb, v, rp_out, ci_out,
                                                          v_out);
    NBP_LAUNCHED();
    return true;
}

static void members_of(const int *map, int n, int nc, int *&mptr, int *&mem, cudaStream_t s);

static Graph coarse_graph(const Graph &G, const int *map, int nc, cudaStream_t s) {
    Graph Gc;
    Gc.n = nc;
    {
        int *mptr = nullptr, *mem = nullptr;
        members_of(map, G.n, nc, mptr, mem, s);
        const bool local = group_rows_local<true>(nc, mptr, mem, G.rp, G.ci, map, 1, 1, G.w, Gc.rp, Gc.ci, Gc.w,
                                                  Gc.nnz, s);
        dfree(mptr, s); dfree(mem, s);
        if (local) return Gc;
    }
    Segments sg = group_by_coarse(G.n, G.nnz, G.rp, G.ci, map, nc, 1, s);
    Gc.nnz = sg.nseg;
    Gc.rp = rowptr_from_segments(sg, nc, s);
    Gc.ci = dmalloc<int>(sg.nseg, s);
    Gc.w = dmalloc<double>(sg.nseg, s);
    if (sg.nseg > 0) {
        k_cg_fill<<<grid_exact(sg.nseg), 256, 0, s>>>(sg.nseg, sg.key, sg.start, sg.nvalid, sg.idx, G.w, (unsigned long long)nc,
                                                      Gc.ci, Gc.w);
        NBP_LAUNCHED();
    }
    free_segments(sg, s);
    return Gc;
}

// 3 passes; agg (n) gets the final map (-1 = isolated); returns the aggregate count
static int aggregate(const DMat &M, double theta, int *agg, cudaStream_t s) {
    const int n = M.nbr, nb = M.bb();
    double *dn = dmalloc<double>(n, s);
    k_diag_norm<<<grid_exact(n), 256, 0, s>>>(n, nb, M.rp, M.ci, M.v, dn);
    NBP_LAUNCHED();
    Graph G;
    G.n = n; G.nnz = M.nnz; G.rp = M.rp; G.ci = M.ci;
    G.w = dmalloc<double>(M.nnz, s);
    k_strength<<<grid_exact(n), 256, 0, s>>>(n, nb, M.rp, M.ci, M.v, dn, G.w);
    NBP_LAUNCHED();
    int *iso = dmalloc<int>(n, s);
    k_isolated<<<grid_exact(n), 256, 0, s>>>(n, M.rp, M.ci, G.w, theta, iso);
    NBP_LAUNCHED();
    dfree(dn, s);
    k_iota<<<grid_exact(n), 256, 0, s>>>(n, agg);
    NBP_LAUNCHED();
    int *map = dmalloc<int>(n, s);
    int nc = n;
    bool own = false;   // the first graph borrows the matrix pattern
    for (int pass = 0; pass < 3; ++pass) {
        const int nn = match_pass(G, theta, map, s);
        k_compose<<<grid_exact(n), 256, 0, s>>>(n, map, agg);
        NBP_LAUNCHED();
        Graph Gc = coarse_graph(G, map, nn, s);
        if (own) graph_free(G, s);
        else dfree(G.w, s);
        G = Gc;
        own = true;
        nc = nn;
    }
    graph_free(G, s);
    dfree(map, s);
    int *keep = dmalloc<int>(nc + 1, s), *newid = dmalloc<int>(nc + 1, s);
    NBP_CUDA(cudaMemsetAsync(keep, 0, sizeof(int) * (nc + 1), s));
    k_mark_keep<<<grid_exact(n), 256, 0, s>>>(n, agg, iso, keep);
    NBP_LAUNCHED();
    exclusive_scan(keep, newid, nc + 1, s);
    const int m = readback(newid + nc, s);
    k_drop_isolated<<<grid_exact(n), 256, 0, s>>>(n, iso, newid, agg);
    NBP_LAUNCHED();
    dfree(keep, s); dfree(newid, s); dfree(iso, s);
    return m;
}

// mptr/mem: the aggregates' member lists (ascending fine index)
static void galerkin(const DMat &M, const int *agg, const int *mptr, const int *mem, int nc, DMat &Mc, cudaStream_t s) {
    Mc = DMat();
    Mc.nbr = nc; Mc.nbc = nc; Mc.br = M.br; Mc.bc = M.bc;
    long long nnz = 0;
    if (group_rows_local<false>(nc, mptr, mem, M.rp, M.ci, agg, 0, M.bb(), M.v, Mc.rp, Mc.ci, Mc.v, nnz, s)) {
        Mc.nnz = nnz;
        return;
    }
    Segments sg = group_by_coarse(M.nbr, M.nnz, M.rp, M.ci, agg, nc, 0, s);
    Mc.nnz = sg.nseg;
    Mc.rp = rowptr_from_segments(sg, nc, s);
    Mc.ci = dmalloc<int>(sg.nseg, s);
    Mc.v = dmalloc<double>((long long)sg.nseg * M.bb(), s);
    if (sg.nseg > 0) {
        k_galerkin_fill<<<grid_exact(sg.nseg), 256, 0, s>>>(sg.nseg, M.bb(), sg.key, sg.start, sg.nvalid, sg.idx, M.v,
                                                            (unsigned long long)nc, Mc.ci, Mc.v);
        NBP_LAUNCHED();
    }
    free_segments(sg, s);
}

// aggregate member lists (ascending fine index) for the restriction
__global__ void k_member_keys(int n, const int *agg, int nc, unsigned int *key, int *val) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    key[i] = agg[i] < 0 ? (unsigned)nc : (unsigned)agg[i];
    val[i] = i;
}
__global__ void k_member_count(int n, const int *agg, int *cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (agg[i] >= 0) atomicAdd(cnt + agg[i], 1);
}

// members of coarse node I (map[i] == I) at mem[mptr[I] .. mptr[I+1]-1],
// ascending; nodes with map < 0 trail
static void members_of(const int *map, int n, int nc, int *&mptr, int *&mem, cudaStream_t s) {
    unsigned int *key = dmalloc<unsigned int>(n, s);
    int *val = dmalloc<int>(n, s);
    k_member_keys<<<grid_exact(n), 256, 0, s>>>(n, map, nc, key, val);
    NBP_LAUNCHED();
    sort_pairs(key, val, n, bits_for((unsigned long long)nc), s);
    int *cnt = dmalloc<int>(nc + 1, s);
    NBP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (nc + 1), s));
    k_member_count<<<grid_exact(n), 256, 0, s>>>(n, map, cnt);
    NBP_LAUNCHED();
    mptr = dmalloc<int>(nc + 1, s);
    exclusive_scan(cnt, mptr, nc + 1, s);
    mem = val;
    dfree(cnt, s); dfree(key, s);
}

static void member_lists(Level &L, int n, int nc, cudaStream_t s) { members_of(L.agg, n, nc, L.mptr, L.mem, s); }

static void dense_inverse(const DMat &M, double *&cinv, int &nc, cudaStream_t s) {
    const int n = M.nbr * M.br;
    nc = n;
    double *Dm = dmalloc<double>((long long)n * n, s);
    cinv = dmalloc<double>((long long)n * n, s);
    NBP_CUDA(cudaMemsetAsync(Dm, 0, sizeof(double) * (size_t)n * n, s));
    k_dense_from_bsr<<<grid_exact(M.nbr), 256, 0, s>>>(M.nbr, M.br, M.rp, M.ci, M.v, Dm);
    k_identity<<<grid_exact((long long)n * n), 256, 0, s>>>(n, cinv);
    NBP_LAUNCHED();
    int *fail = dmalloc<int>(1, s);
    NBP_CUDA(cudaMemsetAsync(fail, 0, sizeof(int), s));
    for (int k = 0; k < n; ++k) {
        k_gj_pivot<<<1, 1024, 0, s>>>(n, k, Dm, cinv, fail);
        k_gj_elim<<<grid_exact((long long)n * 2 * n), 256, 0, s>>>(n, k, Dm, cinv, fail);
        k_gj_clear<<<grid_exact(n), 256, 0, s>>>(n, k, Dm);
    }
    NBP_LAUNCHED();
    const int f = readback(fail, s);
    dfree(fail, s); dfree(Dm, s);
    require(!f, NBP_ERR_INVALID, "setup: coarsest AMG matrix is singular");
}

void amg_build(Hier &H, const DMat &fine, const nbp_options &o, int precision, cudaStream_t s, bool keep_aggregates) {
    // numeric re-setup: the aggregate maps and member lists of the hierarchy
    // H holds are taken over (same pattern); every operator is rebuilt
    int knlev = 0, knc[kMaxLevels] = {};
    int *kagg[kMaxLevels] = {}, *kmptr[kMaxLevels] = {}, *kmem[kMaxLevels] = {};
    if (keep_aggregates) {
        require(H.built && H.nlev >= 1 && H.L[0].M.nbr == fine.nbr && H.L[0].M.nnz == fine.nnz && H.bs == fine.br,
                NBP_ERR_STATE, "setup: no earlier hierarchy of this pattern to build on");
        knlev = H.nlev;
        for (int l = 0; l + 1 < knlev; ++l) {
            kagg[l] = H.L[l].agg; kmptr[l] = H.L[l].mptr; kmem[l] = H.L[l].mem;
            knc[l] = H.L[l + 1].M.nbr;
            H.L[l].agg = nullptr; H.L[l].mptr = nullptr; H.L[l].mem = nullptr;
        }
    }
    auto drop_kept = [&](int from) {
        for (int l = from; l + 1 < knlev; ++l) { dfree(kagg[l], s); dfree(kmptr[l], s); dfree(kmem[l], s); }
    };
    int l = 0;
    try {
        hier_free(H, s);
        H.bs = fine.br;
        // level 0 is a private copy of the fine matrix pattern and values
        DMat &F = H.L[0].M;
        F.nbr = fine.nbr; F.nbc = fine.nbc; F.br = fine.br; F.bc = fine.bc; F.nnz = fine.nnz;
        F.rp = dmalloc<int>(F.nbr + 1, s);
        F.ci = dmalloc<int>(F.nnz, s);
        F.v = dmalloc<double>(F.nnz * F.bb(), s);
        NBP_CUDA(cudaMemcpyAsync(F.rp, fine.rp, sizeof(int) * (F.nbr + 1), cudaMemcpyDeviceToDevice, s));
        NBP_CUDA(cudaMemcpyAsync(F.ci, fine.ci, sizeof(int) * F.nnz, cudaMemcpyDeviceToDevice, s));
        NBP_CUDA(cudaMemcpyAsync(F.v, fine.v, sizeof(double) * F.nnz * F.bb(), cudaMemcpyDeviceToDevice, s));
        const int maxlev = std::max(1, std::min((int)o.amg_max_levels, kMaxLevels));
        while (keep_aggregates ? l + 1 < knlev : (H.L[l].M.nbr > o.amg_coarse_max && l + 1 < maxlev)) {
            Level &L = H.L[l];
            const int n = L.M.nbr;
            int nc;
            if (keep_aggregates) {   // the kept map, now owned by this level
                L.agg = kagg[l]; L.mptr = kmptr[l]; L.mem = kmem[l];
                kagg[l] = kmptr[l] = kmem[l] = nullptr;
                nc = knc[l];
            } else {
                L.agg = dmalloc<int>(n, s);
                nc = aggregate(L.M, o.theta, L.agg, s);
                if (nc >= n || nc == 0) { dfree(L.agg, s); L.agg = nullptr; break; }
                member_lists(L, n, nc, s);
            }
            galerkin(L.M, L.agg, L.mptr, L.mem, nc, H.L[l + 1].M, s);
            ++l;
        }
    } catch (...) {
        drop_kept(0);
        throw;
    }
    H.nlev = l + 1;
    int *singular = dmalloc<int>(1, s);
    NBP_CUDA(cudaMemsetAsync(singular, 0, sizeof(int), s));
    unsigned long long *rb = dmalloc<unsigned long long>(1, s);
    for (int k = 0; k < H.nlev; ++k) {
        Level &L = H.L[k];
        const int n = L.M.nbr, bs = H.bs;
        const long long nv = (long long)n * bs;
        for (int q = 0; q < Level::kWork; ++q) {
            L.w64[q] = dmalloc<double>(nv, s);
            L.w32[q] = dmalloc<float>(nv, s);
        }
        L.kdots = dmalloc<double>(8 + 2 * kKdotBlocks, s);
        NBP_CUDA(cudaMemsetAsync(L.kdots, 0, sizeof(double) * (8 + 2 * kKdotBlocks), s));
        {   // every level, the coarsest included (it is smoothed when too large for a dense solve)
            L.dinv = dmalloc<double>(nv * bs, s);
            k_block_dinv<<<grid_exact(n), 256, 0, s>>>(n, bs, L.M.rp, L.M.ci, L.M.v, L.dinv, singular);
            NBP_CUDA(cudaMemsetAsync(rb, 0, sizeof(unsigned long long), s));
            k_gershgorin<<<grid_exact(n), 256, 0, s>>>(n, bs, L.M.rp, L.M.v, L.dinv, rb);
            NBP_LAUNCHED();
            const unsigned long long bits = readback(rb, s);
            std::memcpy(&L.rho, &bits, sizeof(double));
            if (precision >= 1) {
                L.dinv32 = dmalloc<float>(nv * bs, s);
                k_to_f32<<<grid_for(nv * bs), 256, 0, s>>>(L.dinv, L.dinv32, nv * bs);
                NBP_LAUNCHED();
            }
            make_lowcopies(L.M, precision, s);
            make_sell(L.M, precision, s);
            if (L.M.sl_ci) {   // grids of the sliced kernels, up to 8 threads per row
                L.kpart_blocks = ((long long)L.M.nslice * L.M.sl_c * 8 + 255) / 256;
                L.kpart = dmalloc<double>(2 * L.kpart_blocks, s);
            }
        }
    }
    dfree(rb, s);
    const int sing = readback(singular, s);
    dfree(singular, s);
    require(sing == 0, NBP_ERR_INVALID, "setup: singular diagonal block in an AMG level");
    const Level &C = H.L[H.nlev - 1];
    if ((long long)C.M.nbr * H.bs <= kCoarseDenseMax) {
        dense_inverse(C.M, H.cinv, H.nc, s);
        const long long nn = (long long)H.nc * H.nc;
        H.cinv32 = dmalloc<float>(nn, s);
        k_to_f32<<<grid_for(nn), 256, 0, s>>>(H.cinv, H.cinv32, nn);
        NBP_LAUNCHED();
    } else { H.cinv = nullptr; H.nc = 0; }
    H.built = true;
}

// ================================================================== S_hat
__global__ void k_diagA(int N, const int *rp, const int *ci, const double *v, double *diag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int e = find_entry(rp, ci, i, i);
    for (int a = 0; a < 3; ++a) diag[3 * i + a] = (e >= 0) ? v[(long long)e * 9 + 4 * a] : 0.0;
}
// diag[idx] += r_k (a*a) for outlet k (one launch per outlet: k ascending)
__global__ void k_diagA_lowrank(int beg, int end, const int *oidx, const double *oval, const double *r, int k, double *diag) {
    const int q = beg + blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= end) return;
    const double a = oval[q];
    diag[oidx[q]] = __dadd_rn(diag[oidx[q]], __dmul_rn(r[k], __dmul_rn(a, a)));
}
__global__ void k_recip(long long n, const double *a, double *b) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = 1.0 / a[i];
}
// tuples per row of S_hat: D entries, then C_ik B_kj terms (k ascending, j ascending)
__global__ void k_shat_count(int N, const int *drp, const int *crp, const int *cci, const int *brp, long long *cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    long long c = drp[i + 1] - drp[i];
    for (int e = crp[i]; e < crp[i + 1]; ++e) {
        const int k = cci[e];
        c += brp[k + 1] - brp[k];
    }
    cnt[i] = c;
}
__global__ void k_shat_fill(int N, const int *drp, const int *dci, const int *crp, const int *cci, const double *cv,
                            const int *brp, const int *bci, const double *bv, const double *dinv, const long long *off,
                            unsigned long long *key, double *t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    long long p = off[i];
    for (int e = drp[i]; e < drp[i + 1]; ++e) {
        key[p] = (unsigned long long)i * (unsigned long long)N + (unsigned long long)dci[e];
        t[p++] = 0.0;
    }
    for (int e = crp[i]; e < crp[i + 1]; ++e) {
        const int k = cci[e];
        const double w0 = __dmul_rn(cv[3LL * e], dinv[3LL * k]);
        const double w1 = __dmul_rn(cv[3LL * e + 1], dinv[3LL * k + 1]);
        const double w2 = __dmul_rn(cv[3LL * e + 2], dinv[3LL * k + 2]);
        for (int f = brp[k]; f < brp[k + 1]; ++f) {
            double tt = __dmul_rn(w0, bv[3LL * f]);
            tt = __dadd_rn(tt, __dmul_rn(w1, bv[3LL * f + 1]));
            tt = __dadd_rn(tt, __dmul_rn(w2, bv[3LL * f + 2]));
            key[p] = (unsigned long long)i * (unsigned long long)N + (unsigned long long)bci[f];
            t[p++] = tt;
        }
    }
}
__global__ void k_heads_all(long long n, const unsigned long long *key, int *head) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    head[q] = (q == 0 || key[q - 1] != key[q]) ? 1 : 0;
}
// entry (i, j): s = D_ij (or 0), then s = s - t for each tuple in order
__global__ void k_shat_reduce(int nseg, long long ntup, const unsigned long long *key, const long long *start, const double *t,
                              int N, const int *drp, const int *dci, const double *dv, int *ci_out, double *v_out,
                              int *rowcnt) {
    const int sg = blockIdx.x * blockDim.x + threadIdx.x;
    if (sg >= nseg) return;
    const long long a = start[sg];
    const long long b = (sg + 1 < nseg) ? start[sg + 1] : ntup;
    const unsigned long long k = key[a];
    const int i = (int)(k / (unsigned long long)N), j = (int)(k % (unsigned long long)N);
    const int e = find_entry(drp, dci, i, j);
    double s = (e >= 0) ? dv[e] : 0.0;
    for (long long q = a; q < b; ++q) s = __dsub_rn(s, t[q]);
    ci_out[sg] = j;
    v_out[sg] = s;
    atomicAdd(rowcnt + i, 1);
}

// ---- S_hat one row per warp: the row's tuples (the same as k_shat_fill
// makes, in the same order q) sorted in shared memory by (column, q), so that
// every entry is D_ij minus its terms in order q, as k_shat_reduce sums them;
// for rows of at most kShatRowTuples tuples.
constexpr int kShatRowTuples = 256;
constexpr int kShatWarps = 8;   // warps per block

// Tuples of row i into sk (key = column * 256 + q, padded with ~0u) and, when
// t is set, their terms into t[q].  Returns the tuple count.
__device__ __forceinline__ int shat_row_tuples(int i, int lane, const int *drp, const int *dci, const int *crp,
                                               const int *cci, const double *cv, const int *brp, const int *bci,
                                               const double *bv, const double *dinv, unsigned *sk, double *t) {
    const int d0 = drp[i], dlen = drp[i + 1] - d0;
    const int c0 = crp[i], clen = crp[i + 1] - c0;
    for (int q = lane; q < kShatRowTuples; q += 32) sk[q] = ~0u;
    __syncwarp();
    for (int q = lane; q < dlen; q += 32) {   // the D pattern first, placeholder terms 0
        sk[q] = ((unsigned)dci[d0 + q] << 8) | (unsigned)q;
        if (t) t[q] = 0.0;
    }
    // then C_ik B_kj for k ascending (C's row order), j in B's row order; the
    // start of entry e's tuples is dlen + the B row lengths before it
    int off = dlen;
    for (int e0 = 0; e0 < clen; e0 += 32) {
        const int e = e0 + lane;
        const int k = e < clen ? cci[c0 + e] : 0;
        const int len = e < clen ? brp[k + 1] - brp[k] : 0;
        int incl = len;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int start = off + incl - len;
        if (e < clen) {
            const long long ce = c0 + e;
            double w0 = 0.0, w1 = 0.0, w2 = 0.0;
            if (t) {
                w0 = __dmul_rn(cv[3LL * ce], dinv[3LL * k]);
                w1 = __dmul_rn(cv[3LL * ce + 1], dinv[3LL * k + 1]);
                w2 = __dmul_rn(cv[3LL * ce + 2], dinv[3LL * k + 2]);
            }
            for (int f = 0; f < len; ++f) {
                const int fe = brp[k] + f, q = start + f;
                sk[q] = ((unsigned)bci[fe] << 8) | (unsigned)q;
                if (t) {
                    double tt = __dmul_rn(w0, bv[3LL * fe]);
                    tt = __dadd_rn(tt, __dmul_rn(w1, bv[3LL * fe + 1]));
                    tt = __dadd_rn(tt, __dmul_rn(w2, bv[3LL * fe + 2]));
                    t[q] = tt;
                }
            }
        }
        off += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
    // bitonic sort of the 256 keys (unique: q differs), ascending
    for (int k = 2; k <= kShatRowTuples; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int p = lane; p < kShatRowTuples; p += 32) {
                const int x = p ^ j;
                if (x > p) {
                    const unsigned a = sk[p], b = sk[x];
                    if ((a > b) == ((p & k) == 0)) { sk[p] = b; sk[x] = a; }
                }
            }
            __syncwarp();
        }
    }
    return off;
}

// entries per row (distinct columns)
__global__ void __launch_bounds__(32 * kShatWarps) k_shat_row_count(int N, const int *drp, const int *dci, const int *crp,
                                                                   const int *cci, const int *brp, const int *bci, int *cnt) {
    __shared__ unsigned keys[kShatWarps][kShatRowTuples];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * kShatWarps + w;
    if (i >= N) return;
    unsigned *sk = keys[w];
    const int n = shat_row_tuples(i, lane, drp, dci, crp, cci, nullptr, brp, bci, nullptr, nullptr, sk, nullptr);
    int c = 0;
    for (int p = lane; p < n; p += 32) c += (p == 0 || (sk[p] >> 8) != (sk[p - 1] >> 8)) ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) cnt[i] = c;
}

// the row's entries at rp_out[i]..: columns ascending, each D_ij (or 0)
// minus its terms in order q (as k_shat_reduce)
__global__ void __launch_bounds__(32 * kShatWarps) k_shat_row_fill(int N, const int *drp, const int *dci, const double *dv,
                                                                  const int *crp, const int *cci, const double *cv,
                                                                  const int *brp, const int *bci, const double *bv,
                                                                  const double *dinv, const int *rp_out, int *ci_out,
                                                                  double *v_out) {
    __shared__ unsigned keys[kShatWarps][kShatRowTuples];
    __shared__ double terms[kShatWarps][kShatRowTuples];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * kShatWarps + w;
    if (i >= N) return;
    unsigned *sk = keys[w];
    double *tv = terms[w];
    const int n = shat_row_tuples(i, lane, drp, dci, crp, cci, cv, brp, bci, bv, dinv, sk, tv);
    constexpr int P = kShatRowTuples / 32;   // positions per lane, contiguous
    const int p0 = lane * P;
    bool head[P];
    int mine = 0;
#pragma unroll
    for (int u = 0; u < P; ++u) {
        const int p = p0 + u;
        head[u] = p < n && (p == 0 || (sk[p] >> 8) != (sk[p - 1] >> 8));
        mine += head[u] ? 1 : 0;
    }
    int incl = mine;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    int slot = rp_out[i] + incl - mine;
#pragma unroll
    for (int u = 0; u < P; ++u) {
        if (!head[u]) continue;
        const int p = p0 + u;
        const unsigned j = sk[p] >> 8;
        const int e = find_entry(drp, dci, i, (int)j);
        double sum = (e >= 0) ? dv[e] : 0.0;
        for (int r = p; r < n && (sk[r] >> 8) == j; ++r) sum = __dsub_rn(sum, tv[sk[r] & 255u]);
        ci_out[slot] = (int)j;
        v_out[slot] = sum;
        ++slot;
    }
}

__global__ void k_max_ll(long long n, const long long *a, unsigned long long *out) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) atomicMax(out, (unsigned long long)a[q]);
}

void build_shat(const DMat &A, const DMat &B, const DMat &C, const DMat &D, const LowRank &lr, int N, DMat &S,
                double *diagA_out, cudaStream_t s) {
    double *diag = diagA_out;
    k_diagA<<<grid_exact(N), 256, 0, s>>>(N, A.rp, A.ci, A.v, diag);
    NBP_LAUNCHED();
    for (int k = 0; k < lr.n_out; ++k) {
        int se[2];
        NBP_CUDA(cudaMemcpyAsync(se, lr.optr + k, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        NBP_CUDA(cudaStreamSynchronize(s));
        if (se[1] > se[0]) {
            k_diagA_lowrank<<<grid_exact(se[1] - se[0]), 256, 0, s>>>(se[0], se[1], lr.oidx, lr.oval, lr.r, k, diag);
            NBP_LAUNCHED();
        }
    }
    double *dinv = dmalloc<double>(3LL * N, s);
    k_recip<<<grid_exact(3LL * N), 256, 0, s>>>(3LL * N, diag, dinv);
    long long *cnt = dmalloc<long long>(N + 1, s), *off = dmalloc<long long>(N + 1, s);
    k_shat_count<<<grid_exact(N), 256, 0, s>>>(N, D.rp, C.rp, C.ci, B.rp, cnt);
    NBP_LAUNCHED();
    {   // every row within one warp's sort: the per-row build, no global sort
        unsigned long long *mx = dmalloc<unsigned long long>(1, s);
        NBP_CUDA(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), s));
        k_max_ll<<<grid_exact(N), 256, 0, s>>>(N, cnt, mx);
        NBP_LAUNCHED();
        const unsigned long long maxtup = readback(mx, s);
        dfree(mx, s);
        if (maxtup <= (unsigned long long)kShatRowTuples && N < (1 << 24)) {
            dfree(cnt, s); dfree(off, s);
            int *rowcnt = dmalloc<int>(N + 1, s);
            const unsigned blocks = (unsigned)((N + kShatWarps - 1) / kShatWarps);
            k_shat_row_count<<<blocks, 32 * kShatWarps, 0, s>>>(N, D.rp, D.ci, C.rp, C.ci, B.rp, B.ci, rowcnt);
            NBP_LAUNCHED();
            NBP_CUDA(cudaMemsetAsync(rowcnt + N, 0, sizeof(int), s));
            dmat_free(S, s);
            S.nbr = N; S.nbc = N; S.br = 1; S.bc = 1;
            S.rp = dmalloc<int>(N + 1, s);
            exclusive_scan(rowcnt, S.rp, N + 1, s);
            dfree(rowcnt, s);
            S.nnz = readback(S.rp + N, s);
            S.ci = dmalloc<int>(S.nnz, s);
            S.v = dmalloc<double>(S.nnz, s);
            k_shat_row_fill<<<blocks, 32 * kShatWarps, 0, s>>>(N, D.rp, D.ci, D.v, C.rp, C.ci, C.v, B.rp, B.ci, B.v, dinv,
                                                               S.rp, S.ci, S.v);
            NBP_LAUNCHED();
            dfree(dinv, s);
            return;
        }
    }
    NBP_CUDA(cudaMemsetAsync(cnt + N, 0, sizeof(long long), s));
    exclusive_scan(cnt, off, N + 1, s);
    const long long ntup = readback(off + N, s);
    unsigned long long *key = dmalloc<unsigned long long>(ntup, s);
    double *t = dmalloc<double>(ntup, s);
    k_shat_fill<<<grid_exact(N), 256, 0, s>>>(N, D.rp, D.ci, C.rp, C.ci, C.v, B.rp, B.ci, B.v, dinv, off, key, t);
    NBP_LAUNCHED();
    dfree(cnt, s); dfree(off, s); dfree(dinv, s);
    sort_pairs(key, t, ntup, bits_for((unsigned long long)N * (unsigned long long)N), s);
    int *head = dmalloc<int>(ntup + 1, s), *sid = dmalloc<int>(ntup + 1, s);
    k_heads_all<<<grid_exact(ntup), 256, 0, s>>>(ntup, key, head);
    NBP_LAUNCHED();
    NBP_CUDA(cudaMemsetAsync(head + ntup, 0, sizeof(int), s));
    exclusive_scan(head, sid, ntup + 1, s);
    const int nseg = readback(sid + ntup, s);
    long long *start = dmalloc<long long>(nseg + 1, s);
    k_seg_starts<<<grid_exact(ntup), 256, 0, s>>>(ntup, head, sid, start);
    NBP_LAUNCHED();
    dfree(head, s); dfree(sid, s);
    dmat_free(S, s);
    S.nbr = N; S.nbc = N; S.br = 1; S.bc = 1; S.nnz = nseg;
    S.ci = dmalloc<int>(nseg, s);
    S.v = dmalloc<double>(nseg, s);
    int *rowcnt = dmalloc<int>(N + 1, s);
    NBP_CUDA(cudaMemsetAsync(rowcnt, 0, sizeof(int) * (N + 1), s));
    k_shat_reduce<<<grid_exact(nseg), 256, 0, s>>>(nseg, ntup, key, start, t, N, D.rp, D.ci, D.v, S.ci, S.v, rowcnt);
    NBP_LAUNCHED();
    S.rp = dmalloc<int>(N + 1, s);
    exclusive_scan(rowcnt, S.rp, N + 1, s);
    dfree(rowcnt, s); dfree(key, s); dfree(t, s); dfree(start, s);
}

// ============================================================== transpose
__global__ void k_tr_keys(int n, const int *rp, const int *ci, unsigned int *key, int *val) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int e = rp[i]; e < rp[i + 1]; ++e) { key[e] = (unsigned)ci[e]; val[e] = e; }
}
__global__ void k_tr_count(long long nnz, const int *ci, int *cnt) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nnz) atomicAdd(cnt + ci[e], 1);
}
__global__ void k_tr_fill(long long nnz, int br, int bc, const int *row, const int *perm, const double *v, int *ci_out,
                          double *v_out) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nnz) return;
    const int e = perm[p];
    ci_out[p] = row[e];
    const double *src = v + (long long)e * br * bc;
    double *dst = v_out + p * br * bc;
    for (int a = 0; a < br; ++a)
        for (int b = 0; b < bc; ++b) dst[b * br + a] = src[a * bc + b];
}

// out = in^T (blocks transposed); rows of out sorted by column (stable sort)
void transpose_dmat(const DMat &in, DMat &out, cudaStream_t s) {
    dmat_free(out, s);
    out.nbr = in.nbc; out.nbc = in.nbr; out.br = in.bc; out.bc = in.br; out.nnz = in.nnz;
    unsigned int *key = dmalloc<unsigned int>(in.nnz, s);
    int *perm = dmalloc<int>(in.nnz, s);
    k_tr_keys<<<grid_exact(in.nbr), 256, 0, s>>>(in.nbr, in.rp, in.ci, key, perm);
    NBP_LAUNCHED();
    sort_pairs(key, perm, in.nnz, bits_for((unsigned long long)in.nbc), s);
    int *row = dmalloc<int>(in.nnz, s);
    k_entry_rows<<<grid_exact(in.nbr), 256, 0, s>>>(in.nbr, in.rp, row);
    int *cnt = dmalloc<int>(out.nbr + 1, s);
    NBP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (out.nbr + 1), s));
    k_tr_count<<<grid_exact(in.nnz), 256, 0, s>>>(in.nnz, in.ci, cnt);
    NBP_LAUNCHED();
    out.rp = dmalloc<int>(out.nbr + 1, s);
    exclusive_scan(cnt, out.rp, out.nbr + 1, s);
    out.ci = dmalloc<int>(out.nnz, s);
    out.v = dmalloc<double>(out.nnz * out.bb(), s);
    k_tr_fill<<<grid_exact(in.nnz), 256, 0, s>>>(in.nnz, in.br, in.bc, row, perm, in.v, out.ci, out.v);
    NBP_LAUNCHED();
    dfree(key, s); dfree(perm, s); dfree(row, s); dfree(cnt, s);
}

}  // namespace nbp
