// solver.cu -- the nested block preconditioned solve on one GB300 and its C ABI.
//
//   outer   FGMRES(m), FP64, right preconditioned by P_SCR      (paper Sec. 3)
//   P_SCR   Algorithm 3: A-solve, C product, S-solve, B product, A-solve
//   S x     Algorithm 2: D x - C A^{-1} B x with an inner A-solve (delta_I)
//   A-solve GMRES(m_A) with P_A = aggregation AMG V(1,1) (or Jacobi)
//   S-solve GMRES(m_S) with P_S = AMG(S_hat), S_hat = D - C diag(A)^{-1} B
//
// Every level runs the flexible form of GMRES (the preconditioned directions
// Z are stored), which equals right-preconditioned GMRES for a fixed linear
// preconditioner and saves the final preconditioner application.  Arnoldi is
// classical Gram-Schmidt with one re-orthogonalisation (CGS2) on fused
// multi-dot / multi-axpy kernels with fixed-order reductions, so a run is
// bitwise repeatable.  The Givens update runs on the device; the host reads a
// 24-byte status per iteration to decide convergence.
//
// Precision modes: 0 = FP64 throughout; 1 = the intermediate/inner solves
// (Algorithms 2-3 and below) in FP32 values, vectors and Krylov basis; 2 = as
// 1 with BF16 matrix values.  The outer FGMRES, its Givens update, the true
// residual and the rank-one resistance term stay FP64; the flexible outer
// iteration absorbs the inexact preconditioner (Sec. 3: the preconditioner
// may vary between iterations).
#include <chrono>
#include <cmath>
#include <cstring>
#include <algorithm>
#include <numeric>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>

#include "kernels.cuh"
#include "spmv.cuh"
#include "rcr.cuh"
#include "vms.cuh"

namespace nbp {

// ------------------------------------------------------------ profiling
struct Prof {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    struct Rec { int cat; size_t e0; double bytes; std::string tag; };
    std::vector<Rec> recs;
    long long launches = 0;
    cudaEvent_t get() {
        if (used == pool.size()) {
            cudaEvent_t e;
            NBP_CUDA(cudaEventCreate(&e));
            pool.push_back(e);
        }
        return pool[used++];
    }
    ~Prof() {
        for (auto e : pool) cudaEventDestroy(e);
    }
};
enum { CAT_SPMV = 0, CAT_SPMV_A0 = 1, CAT_ARNOLDI = 2, CAT_VCYCLE = 3, CAT_CHEB_A0 = 4, CAT_OTHER = 5 };

// ------------------------------------------------------------ Krylov space
template <typename T> struct Krylov {
    long long n = 0, ld = 0;   // basis columns at V + j*ld, ld = n rounded up to 32 (128-byte columns)
    int m = 0;
    T *V = nullptr, *Z = nullptr, *w = nullptr, *r = nullptr;
    double *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr;
    double *h1 = nullptr, *h2 = nullptr, *nrm = nullptr, *beta = nullptr, *partial = nullptr;
    unsigned *ticket = nullptr;   // last-block ticket of the Arnoldi reductions
    GmState *st = nullptr;
    // blocks of the Gram-Schmidt reductions, autotuned per n (0: one wave):
    // grid_md for the first multi-dot of a step, which meets the basis cold
    // (the preconditioner's sweeps have evicted it from L2), grid for the
    // fused subtract + products passes that follow it on the same columns
    unsigned grid = 0, grid_md = 0;
    void ensure(long long n_, int m_, cudaStream_t s) {
        if (n_ == n && m_ <= m) return;
        const unsigned keep_grid = (n_ == n) ? grid : 0u, keep_md = (n_ == n) ? grid_md : 0u;
        release(s);
        grid = keep_grid;
        grid_md = keep_md;
        n = n_; m = m_;
        ld = (n + 31) / 32 * 32;
        V = dmalloc<T>((size_t)ld * (m + 1), s);
        Z = dmalloc<T>((size_t)ld * m, s);
        w = dmalloc<T>(n, s);
        r = dmalloc<T>(n, s);
        H = dmalloc<double>((size_t)(m + 1) * m, s);
        cs = dmalloc<double>(m, s); sn = dmalloc<double>(m, s);
        g = dmalloc<double>(m + 1, s); y = dmalloc<double>(m, s);
        h1 = dmalloc<double>(m + 1, s); h2 = dmalloc<double>(m + 1, s);
        nrm = dmalloc<double>(1, s); beta = dmalloc<double>(1, s);
        partial = dmalloc<double>((size_t)kReduceBlocks * (m + 1), s);
        ticket = dmalloc<unsigned>(1, s);
        NBP_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned), s));
        st = dmalloc<GmState>(1, s);
    }
    void release(cudaStream_t s) {
        dfree(V, s); dfree(Z, s); dfree(w, s); dfree(r, s); dfree(H, s); dfree(cs, s); dfree(sn, s); dfree(g, s);
        dfree(y, s); dfree(h1, s); dfree(h2, s); dfree(nrm, s); dfree(beta, s); dfree(partial, s); dfree(ticket, s);
        dfree(st, s);
        *this = Krylov();
    }
    GivensArgs givens(int j) const {
        GivensArgs q;
        q.H = H; q.ldh = m; q.j = j; q.h1 = h1; q.h2 = h2; q.cs = cs; q.sn = sn; q.g = g; q.st = st;
        return q;
    }
};

template <typename T> struct Bufs {   // vectors of Algorithms 2-3 in the inner type
    long long N = 0;
    T *sv = nullptr, *sp = nullptr, *yvh = nullptr, *sp2 = nullptr, *yp = nullptr, *sv2 = nullptr, *yv = nullptr;
    T *xbar = nullptr, *xtil = nullptr, *dinvA = nullptr;
    void ensure(long long N_, cudaStream_t s) {
        if (N_ == N) return;
        release(s);
        N = N_;
        sv = dmalloc<T>(3 * N, s); sp = dmalloc<T>(N, s); yvh = dmalloc<T>(3 * N, s); sp2 = dmalloc<T>(N, s);
        yp = dmalloc<T>(N, s); sv2 = dmalloc<T>(3 * N, s); yv = dmalloc<T>(3 * N, s);
        xbar = dmalloc<T>(3 * N, s); xtil = dmalloc<T>(3 * N, s); dinvA = dmalloc<T>(3 * N, s);
    }
    void release(cudaStream_t s) {
        dfree(sv, s); dfree(sp, s); dfree(yvh, s); dfree(sp2, s); dfree(yp, s); dfree(sv2, s); dfree(yv, s);
        dfree(xbar, s); dfree(xtil, s); dfree(dinvA, s);
        *this = Bufs();
    }
};

}  // namespace nbp

// ------------------------------------------------------------------ context
struct nbp_ctx {
    int dev = 0;
    cudaStream_t s = nullptr;
    int N = 0;
    nbp::DMat A, B, C, D, Shat;
    nbp::LowRank lr;
    nbp_options opt{};
    nbp::Hier HA, HS;
    double *diagA = nullptr;      // scalar diagonal of A incl. rank-one terms (3N)
    bool setup_done = false;
    int setup_precision = -1;
    double setup_s = 0.0;
    nbp::Krylov<double> Kout, KA64, KS64;
    nbp::Krylov<float> KA32, KS32;
    nbp::Bufs<double> B64;
    nbp::Bufs<float> B32;
    double *full_w = nullptr;     // 4N scratch of the outer operator
    double *rcr_buf = nullptr;    // RCR update: Q, m and the new weights when the caller keeps none (3 n_out)
    int *rcr_bad = nullptr;       // RCR update: non-finite m^k seen
    nbp::GmState *hst = nullptr;  // pinned host status
    nbp_info info{};
    nbp::Prof prof;
    nbp_profile_info pinfo{};
    std::string err;
    std::string report;
    nbp_ctx *tctx = nullptr;      // transposed system (adjoint), built lazily
    bool is_transposed = false;
    // CUDA graphs of the AMG cycles, keyed by (hierarchy, value precision, Chebyshev degree)
    struct CycleGraph { cudaGraphExec_t exec = nullptr; int cheb = -1; long long kernels = 0; };
    static constexpr int kMaxChebDegree = 8;
    // inside an inner A-solve of Algorithm 2 with gs_passes_I = 1: one
    // classical Gram-Schmidt pass per Arnoldi step instead of two
    bool gs_one_pass = false;
    CycleGraph graphs[2][3][kMaxChebDegree + 1];
    cudaStream_t cap = nullptr;   // private stream used only while capturing
    bool use_graphs = true;
    // device-driven solve: the whole nested solve as one CUDA graph whose
    // Krylov loops are graph WHILE nodes (dl_st: loop states of the outer,
    // S and A levels; dl_par: per-solve options; dl_cnt: iteration counters;
    // dl_b, dl_x: its fixed right-hand side and solution; dl_zo: the outer
    // preconditioned vector; dl_zA, dl_zS: preconditioner outputs when the
    // preconditioner is not an AMG cycle; dl_cap: capture streams by loop depth)
    nbp::GmDev *dl_st = nullptr;
    nbp::DlParams *dl_par = nullptr;
    nbp::DlCounters *dl_cnt = nullptr;
    double *dl_b = nullptr, *dl_x = nullptr, *dl_zo = nullptr;
    void *dl_zA = nullptr, *dl_zS = nullptr;
    nbp::DlParams dl_hpar{};               // host copy of the per-solve options (source of the upload)
    nbp::GmDev *dl_host = nullptr;         // pinned copy of the outer loop state
    nbp::DlCounters *dl_hcnt = nullptr;    // pinned copy of the counters
    cudaStream_t dl_cap[4] = {};
    cudaGraphExec_t dl_exec = nullptr;     // the single-solve graph
    // kernel nodes of the captured solve, to count the kernels one solve runs:
    // outside every loop, per restart cycle, per outer iteration, per A- or
    // I-iteration, per S-iteration (nested loops' bodies not included)
    long long dl_k_top = 0, dl_k_cycle = 0, dl_k_outer = 0, dl_k_A = 0, dl_k_S = 0;
    unsigned long long graph_gen = 0;      // bumped whenever captured graphs go stale
    std::vector<const void *> dl_key;      // buffers and options the graph was captured with
};

namespace nbp {

// ------------------------------------------------------------ small helpers
// value copy of the inner operators (0 FP64, 1 FP32, 2 BF16) per precision mode
static inline int vsel_of(int precision) { return precision == 2 ? 2 : (precision >= 1 ? 1 : 0); }
// value copy of the AMG hierarchies: BF16 in modes 2-4
static inline int amg_vsel_of(int precision) { return precision >= 2 ? 2 : (precision == 1 ? 1 : 0); }
// copies a precision mode needs built at setup (modes 2-4 need the same)
static inline int build_level(int precision) { return precision >= 2 ? 2 : precision; }
// value copy of A in the inner A-solves of Algorithm 2 (the S-apply's
// A^{-1}, tolerance rtol_I): mode 4 applies A there with BF16 values
static inline int vsel_I_of(int precision) { return precision == 4 ? 2 : vsel_of(precision); }

template <typename T> static void fill(T *x, T v, long long n, cudaStream_t s) {
    k_fill<T><<<grid_for(n), 256, 0, s>>>(x, v, n);
    NBP_LAUNCHED();
}
template <typename D_, typename S_> static void convert(D_ *d, const S_ *src, long long n, cudaStream_t s) {
    k_convert<D_, S_><<<grid_for(n), 256, 0, s>>>(d, src, n);
    NBP_LAUNCHED();
}
template <typename T> static void copy(T *d, const T *src, long long n, cudaStream_t s) {
    NBP_CUDA(cudaMemcpyAsync(d, src, sizeof(T) * n, cudaMemcpyDeviceToDevice, s));
}

static void prof_begin(nbp_ctx *c, cudaEvent_t &e) {
    c->prof.launches++;
    if (!c->prof.on) return;
    e = c->prof.get();
    NBP_CUDA(cudaEventRecord(e, c->s));
}
static void prof_end(nbp_ctx *c, int cat, double bytes, const std::string &tag = std::string()) {
    if (!c->prof.on) return;
    cudaEvent_t e1 = c->prof.get();
    NBP_CUDA(cudaEventRecord(e1, c->s));
    c->prof.recs.push_back({cat, c->prof.used - 2, bytes, tag});
}

// launch f() with event timing under `tag` when profiling (small kernels)
template <class F> static void timed(nbp_ctx *c, const char *tag, double bytes, F f) {
    cudaEvent_t e0;
    prof_begin(c, e0);
    f();
    NBP_LAUNCHED();
    prof_end(c, CAT_OTHER, bytes, tag);
}

static std::string mat_tag(nbp_ctx *c, const DMat &M, int epi) {
    static const char *en[] = {"set", "add", "sub", "res", "cheb"};
    std::string t;
    if (&M == &c->A) t = "A";
    else if (&M == &c->B) t = "B";
    else if (&M == &c->C) t = "C";
    else if (&M == &c->D) t = "D";
    else {
        for (int l = 0; l < c->HA.nlev && t.empty(); ++l)
            if (&M == &c->HA.L[l].M) t = "HA" + std::to_string(l);
        for (int l = 0; l < c->HS.nlev && t.empty(); ++l)
            if (&M == &c->HS.L[l].M) t = "HS" + std::to_string(l);
        if (t.empty()) t = "M";
    }
    const int kind = M.tuned >= 0 ? M.tuned : (M.sl_ci ? 0 : -1);
    const std::string k = kind == 0 ? "/sell" + std::to_string(M.sl_c)
                          : is_sellm(kind) ? "/sell" + std::to_string(M.sl_c) + "x" + std::to_string(kind - kSellMT)
                                           : "/flat" + std::to_string(kind);
    return t + "/" + en[epi] + k;
}

// extra_bytes: algorithmic bytes of a fused epilogue that the product's own
// count leaves out (the rank-one term)
template <typename XT>
static void do_spmv(nbp_ctx *c, const DMat &M, int vsel, SpmvArgs a, int epi, bool lr, int cat = CAT_SPMV,
                    double extra_bytes = 0.0) {
    cudaEvent_t e0;
    prof_begin(c, e0);
    const double bytes = spmv<XT>(M, vsel, a, epi, lr, c->s) + extra_bytes;
    prof_end(c, cat, bytes, c->prof.on ? mat_tag(c, M, epi) : std::string());
}

static SpmvArgs sargs(const void *x, void *y) {
    SpmvArgs a{};
    a.x = x;
    a.y = y;
    return a;
}

// Run f as an inner A-solve of Algorithm 2: the AMG(A) cycle of degree
// cheb_degree_I (the hierarchy's own degree, cheb_degree, everywhere else)
// and gs_passes_I Gram-Schmidt passes per Arnoldi step (two elsewhere)
template <class F> static void as_inner_solve(nbp_ctx *c, F f) {
    const int keep = c->HA.cheb;
    const bool keep1 = c->gs_one_pass;
    c->HA.cheb = c->opt.cheb_degree_I;
    c->gs_one_pass = c->opt.gs_passes_I == 1;
    try {
        f();
    } catch (...) {
        c->HA.cheb = keep;
        c->gs_one_pass = keep1;
        throw;
    }
    c->HA.cheb = keep;
    c->gs_one_pass = keep1;
}

// y = A x (+ sum_k r_k a^k (a^k . x)); the rank-one factors f_k are FP64
template <typename T> static void apply_A(nbp_ctx *c, int vsel, const T *x, T *y) {
    LowRank &lr = c->lr;
    SpmvArgs a = sargs(x, y);
    if (lr.n_out > 0) {
        c->prof.launches++;
        k_lowrank_dots<T><<<lr.n_out, 256, 0, c->s>>>(lr.optr, lr.oidx, lr.oval, lr.r, x, lr.f);
        NBP_LAUNCHED();
        a.lr_rp = lr.lr_rp; a.lr_k = lr.lr_k; a.lr_c = lr.lr_c; a.lr_val = lr.lr_val; a.lr_f = lr.f;
    }
    // rank-one epilogue: the per-row list pointers, each (outlet, component,
    // value) entry once and the n_out factors
    const double lr_bytes = lr.n_out > 0 ? (double)(c->N + 1) * 4.0 + (double)lr.no * 16.0 + lr.n_out * 8.0 : 0.0;
    do_spmv<T>(c, c->A, vsel, a, EPI_SET, lr.n_out > 0, CAT_SPMV_A0, lr_bytes);
}

// ------------------------------------------------------------ CGS2 Arnoldi
static inline bool al16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// One wave of the fixed-grid kernel: kSMs x (resident blocks per SM, at most
// 4), so that no block waits for a second wave; fixed per kernel, so the
// partial sums keep one order.
template <typename F> static unsigned one_wave(F kernel) {
    int per_sm = 0;
    NBP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0));
    return (unsigned)(kSMs * std::max(1, std::min(4, per_sm)));
}


// out = V(:, 0..ncols-1)^T w, reduced on the device by the grid's last block
// (which also applies the Givens update gv when gv.H is set)
constexpr int kFusedCols = 16;   // longest basis of the fused subtract + products kernel

// grids of the fixed-grid Arnoldi kernels, taken once per kernel (and before
// any graph capture: see dl_prepare)
template <typename T> struct ArnoldiGrids {
    unsigned mdot_v, mdot_s, mdot_dl_v, mdot_dl_s, mpd_dl_v, mpd_dl_s;
};
template <typename T> static const ArnoldiGrids<T> &arnoldi_grids() {
    static const ArnoldiGrids<T> g = {one_wave(k_mdot<T, 8, true>), one_wave(k_mdot<T, 8, false>),
                                      one_wave(k_mdot_dl<T, 8, true>), one_wave(k_mdot_dl<T, 8, false>),
                                      one_wave(k_maxpy_dot_dl<T, kFusedCols, true>),
                                      one_wave(k_maxpy_dot_dl<T, kFusedCols, false>)};
    return g;
}

template <typename T> static void mdot(nbp_ctx *c, Krylov<T> &K, const T *V, long long ldv, int ncols, const T *w, double *out,
                                       GivensArgs gv = GivensArgs()) {
    cudaEvent_t e0;
    prof_begin(c, e0);
    const bool vec = al16(V) && al16(w) && (ncols <= 1 || (ldv * (long long)sizeof(T)) % 16 == 0);
    const unsigned g1 = K.grid_md ? K.grid_md : arnoldi_grids<T>().mdot_v, g0 = K.grid_md ? K.grid_md : arnoldi_grids<T>().mdot_s;
    if (vec) k_mdot<T, 8, true><<<g1, 256, 0, c->s>>>(V, ldv, ncols, w, K.n, K.partial, out, K.ticket, gv);
    else k_mdot<T, 8, false><<<g0, 256, 0, c->s>>>(V, ldv, ncols, w, K.n, K.partial, out, K.ticket, gv);
    NBP_LAUNCHED();
    prof_end(c, CAT_ARNOLDI, (double)(ncols + 1) * K.n * sizeof(T), "arnoldi/mdot");
}
template <typename T> static void maxpy(nbp_ctx *c, long long n, const T *V, long long ldv, int ncols, const double *coef,
                                        double alpha, T *w) {
    cudaEvent_t e0;
    prof_begin(c, e0);
    const bool vec = al16(V) && al16(w) && (ncols <= 1 || (ldv * (long long)sizeof(T)) % 16 == 0);
    const unsigned grid = grid_for(n / (vec ? Vec16<T>::W : 1) + 1, 256, 8LL * kSMs * 4);
    if (vec) k_maxpy<T, true><<<grid, 256, 0, c->s>>>(V, ldv, ncols, coef, alpha, w, n);
    else k_maxpy<T, false><<<grid, 256, 0, c->s>>>(V, ldv, ncols, coef, alpha, w, n);
    NBP_LAUNCHED();
    prof_end(c, CAT_ARNOLDI, (double)(ncols + 2) * n * sizeof(T), "arnoldi/maxpy");
}

template <typename T, int MAXC, bool VEC>
static void launch_maxpy_dot_v(nbp_ctx *c, Krylov<T> &K, const T *V, long long ldv, int ncols, const double *coef, T *w,
                               int norm_only, double *out, GivensArgs gv) {
    static const unsigned wave = one_wave(k_maxpy_dot<T, MAXC, VEC>);
    const unsigned grid = K.grid ? K.grid : wave;
    k_maxpy_dot<T, MAXC, VEC><<<grid, 256, 0, c->s>>>(V, ldv, ncols, coef, w, K.n, norm_only, K.partial, out, K.ticket, gv);
}
template <typename T, int MAXC>
static void launch_maxpy_dot(nbp_ctx *c, Krylov<T> &K, bool vec, const T *V, long long ldv, int ncols, const double *coef,
                             T *w, int norm_only, double *out, GivensArgs gv) {
    if (vec) launch_maxpy_dot_v<T, MAXC, true>(c, K, V, ldv, ncols, coef, w, norm_only, out, gv);
    else launch_maxpy_dot_v<T, MAXC, false>(c, K, V, ldv, ncols, coef, w, norm_only, out, gv);
}

// w -= V coef (ncols <= kFusedCols columns), then out = V^T w (or ||w||^2
// when norm_only, followed by the Givens update gv), in one pass over V
template <typename T> static void maxpy_dot(nbp_ctx *c, Krylov<T> &K, const T *V, long long ldv, int ncols,
                                            const double *coef, T *w, int norm_only, double *out,
                                            GivensArgs gv = GivensArgs()) {
    cudaEvent_t e0;
    prof_begin(c, e0);
    const bool vec = al16(V) && al16(w) && (ncols <= 1 || (ldv * (long long)sizeof(T)) % 16 == 0);
    if (ncols <= 4) launch_maxpy_dot<T, 4>(c, K, vec, V, ldv, ncols, coef, w, norm_only, out, gv);
    else if (ncols <= 8) launch_maxpy_dot<T, 8>(c, K, vec, V, ldv, ncols, coef, w, norm_only, out, gv);
    else launch_maxpy_dot<T, kFusedCols>(c, K, vec, V, ldv, ncols, coef, w, norm_only, out, gv);
    NBP_LAUNCHED();
    prof_end(c, CAT_ARNOLDI, (double)(ncols + 2) * K.n * sizeof(T), "arnoldi/maxpy_dot");
}

template <typename T> static void scale_inv(nbp_ctx *c, T *v, const T *w, const double *sc, long long n) {
    const bool vec = al16(v) && al16(w);
    const unsigned grid = grid_for(n / (vec ? Vec16<T>::W : 1) + 1);
    if (vec) k_scale_inv<T, true><<<grid, 256, 0, c->s>>>(v, w, sc, n);
    else k_scale_inv<T, false><<<grid, 256, 0, c->s>>>(v, w, sc, n);
}

// Autotuner of the Gram-Schmidt kernels' grids for one vector length: the
// candidates (one wave, a half and a quarter of it, a quarter block per SM,
// just enough blocks for eight 16-byte pieces per thread, and kReduceBlocks
// and half of it, capped at a block per 256 pieces) are timed on a
// four-column step in the space's own buffers, as the solve meets it: the
// multi-dot after a write of a buffer larger than L2 (between two steps the
// preconditioner's sweeps evict the basis), then the subtract + products and
// subtract + norm passes on the columns it left in L2.  Three batches of
// five steps; each kernel keeps its own fastest grid.  A short vector leaves
// most of a one-wave grid idle in its reductions (what a batch of small
// instances meets), while a cold pass over a long one needs every block's
// loads in flight.  The choice is cached per (vector length, type) for the
// life of the process, so every space of that length sums in the same order.
static std::mutex g_arnoldi_tune_mutex;
static std::map<std::pair<long long, int>, std::pair<unsigned, unsigned>> g_arnoldi_tune;

template <typename T> static void tune_arnoldi(nbp_ctx *c, Krylov<T> &K) {
    if (K.grid || K.m < 4 || c->prof.on) return;
    const auto key = std::make_pair(K.n, (int)sizeof(T));
    {
        std::lock_guard<std::mutex> lock(g_arnoldi_tune_mutex);
        auto it = g_arnoldi_tune.find(key);
        if (it != g_arnoldi_tune.end()) { K.grid = it->second.first; K.grid_md = it->second.second; return; }
    }
    const bool vec = al16(K.V) && al16(K.w) && (K.ld * (long long)sizeof(T)) % 16 == 0;
    const ArnoldiGrids<T> &ag = arnoldi_grids<T>();
    static const unsigned w4v = one_wave(k_maxpy_dot<T, 4, true>), w4s = one_wave(k_maxpy_dot<T, 4, false>);
    unsigned gmax = vec ? std::min({ag.mdot_v, ag.mdot_dl_v, ag.mpd_dl_v, w4v})
                        : std::min({ag.mdot_s, ag.mdot_dl_s, ag.mpd_dl_s, w4s});
    gmax = std::max(1u, std::min(gmax, (unsigned)kReduceBlocks));
    const long long pieces = (K.n + Vec16<T>::W - 1) / Vec16<T>::W;
    // also grids of several waves of the lowest-occupancy kernel, up to the
    // partial buffers' kReduceBlocks: any grid sums correctly (fixed chunks,
    // last-block reduction), and a long vector streams faster with more
    // blocks than one wave of the widest kernel holds
    const unsigned gbig = (unsigned)std::min<long long>(kReduceBlocks, std::max<long long>(1, pieces / 256));
    std::vector<unsigned> cands = {gmax, gmax / 2, gmax / 4, (unsigned)kSMs / 4,
                                   (unsigned)std::min<long long>(gmax, (pieces + 8 * 256 - 1) / (8 * 256)),
                                   gbig, gbig / 2};
    std::sort(cands.begin(), cands.end());
    cands.erase(std::unique(cands.begin(), cands.end()), cands.end());
    constexpr size_t kFlush = 256ull << 20;   // twice the L2
    char *flush = dmalloc<char>(kFlush, c->s);
    fill<T>(K.V, T(1), (long long)K.ld * 4, c->s);
    fill<T>(K.w, T(1), K.n, c->s);
    NBP_CUDA(cudaMemsetAsync(K.h1, 0, sizeof(double) * 4, c->s));
    cudaEvent_t ev[3];
    for (cudaEvent_t &e : ev) NBP_CUDA(cudaEventCreate(&e));
    float best = 1e30f, best_md = 1e30f;
    unsigned arg = gmax, arg_md = gmax;
    const long long launches = c->prof.launches;
    for (unsigned g : cands) {
        if (g == 0) continue;
        K.grid = K.grid_md = g;
        float tb = 1e30f, tb_md = 1e30f;
        for (int r = 0; r < 3; ++r) {
            float t = 0.f, t_md = 0.f;
            for (int q = 0; q < 5; ++q) {
                NBP_CUDA(cudaMemsetAsync(flush, (r * 5 + q) & 0xff, kFlush, c->s));
                NBP_CUDA(cudaEventRecord(ev[0], c->s));
                mdot<T>(c, K, K.V, K.ld, 4, K.w, K.h2);
                NBP_CUDA(cudaEventRecord(ev[1], c->s));
                maxpy_dot<T>(c, K, K.V, K.ld, 4, K.h1, K.w, 0, K.h2);
                maxpy_dot<T>(c, K, K.V, K.ld, 4, K.h1, K.w, 1, K.nrm);
                NBP_CUDA(cudaEventRecord(ev[2], c->s));
                NBP_CUDA(cudaEventSynchronize(ev[2]));
                float a = 0.f, b = 0.f;
                NBP_CUDA(cudaEventElapsedTime(&a, ev[0], ev[1]));
                NBP_CUDA(cudaEventElapsedTime(&b, ev[1], ev[2]));
                t_md += a;
                t += b;
            }
            tb = std::min(tb, t);
            tb_md = std::min(tb_md, t_md);
        }
        if (tb < best) { best = tb; arg = g; }
        if (tb_md < best_md) { best_md = tb_md; arg_md = g; }
    }
    c->prof.launches = launches;
    for (cudaEvent_t &e : ev) cudaEventDestroy(e);
    dfree(flush, c->s);
    std::lock_guard<std::mutex> lock(g_arnoldi_tune_mutex);
    auto it = g_arnoldi_tune.find(key);
    if (it != g_arnoldi_tune.end()) { arg = it->second.first; arg_md = it->second.second; }
    else g_arnoldi_tune[key] = std::make_pair(arg, arg_md);
    K.grid = arg;
    K.grid_md = arg_md;
}

// ----------------------------------------------------------------- GMRES
struct GmResult { int its = 0; double rel = 0.0, rel_true = -1.0; int conv = 0; };

static void read_state(nbp_ctx *c, const GmState *st) {
    NBP_CUDA(cudaMemcpyAsync(c->hst, st, sizeof(GmState), cudaMemcpyDeviceToHost, c->s));
    const auto t0 = std::chrono::steady_clock::now();
    NBP_CUDA(cudaStreamSynchronize(c->s));
    c->pinfo.host_wait_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    c->pinfo.host_syncs++;
}

// Restarted flexible GMRES, x_0 = 0; stops when the residual estimate
// |g_{j+1}| <= max(rtol ||b||, atol) (confirmed on the true residual when
// check_true) or after nmax iterations.
template <typename T, typename Op, typename Pc>
static GmResult gmres(nbp_ctx *c, Krylov<T> &K, long long n, Op op, Pc pc, const T *b, T *x, double rtol, double atol,
                      int m, int nmax, bool check_true) {
    cudaStream_t s = c->s;
    GmResult R;
    m = std::max(1, std::min(m, std::max(nmax, 1)));
    K.ensure(n, m, s);
    tune_arnoldi<T>(c, K);
    fill<T>(x, T(0), n, s);
    mdot<T>(c, K, b, n, 1, b, K.nrm);
    c->prof.launches++;
    k_gm_init<<<1, 256, 0, s>>>(K.g, m + 1, K.nrm, K.beta, K.st);
    NBP_LAUNCHED();
    read_state(c, K.st);
    const double bnorm = c->hst->res;
    require(std::isfinite(bnorm), NBP_ERR_NAN, "gmres: right-hand side is not finite");
    const double tol = std::max(rtol * bnorm, atol);
    double res = bnorm;
    R.rel_true = bnorm > 0 ? 1.0 : 0.0;
    if (bnorm <= tol) { R.conv = 1; R.rel = bnorm > 0 ? res / bnorm : 0.0; return R; }
    const T *r0 = b;   // first cycle: r = b (x_0 = 0)
    while (R.its < nmax) {
        c->prof.launches++;
        scale_inv<T>(c, K.V, r0, K.beta, n);
        NBP_LAUNCHED();
        int jend = 0;
        for (int j = 0; j < m && R.its < nmax; ++j) {
            T *vj = K.V + (size_t)j * K.ld, *zj = K.Z + (size_t)j * K.ld;
            pc(vj, zj);
            // CGS2: two Gram-Schmidt passes against V(:, 0..j); the first
            // inner products ride on the operator when it can, and for short
            // bases each subtraction is fused with the next inner products
            op(zj, K.w);
            mdot<T>(c, K, K.V, K.ld, j + 1, K.w, K.h1);
            // second pass; the last kernel also forms ||w|| and applies the
            // Givens update of column j on the device
            if (c->gs_one_pass) {   // one pass: subtract, norm and Givens update
                GivensArgs gv = K.givens(j);
                gv.h2 = nullptr;
                if (j + 1 <= kFusedCols) {
                    maxpy_dot<T>(c, K, K.V, K.ld, j + 1, K.h1, K.w, 1, K.nrm, gv);
                } else {
                    maxpy<T>(c, n, K.V, K.ld, j + 1, K.h1, -1.0, K.w);
                    mdot<T>(c, K, K.w, K.ld, 1, K.w, K.nrm, gv);
                }
            } else if (j + 1 <= kFusedCols) {
                maxpy_dot<T>(c, K, K.V, K.ld, j + 1, K.h1, K.w, 0, K.h2);
                maxpy_dot<T>(c, K, K.V, K.ld, j + 1, K.h2, K.w, 1, K.nrm, K.givens(j));
            } else {
                maxpy<T>(c, n, K.V, K.ld, j + 1, K.h1, -1.0, K.w);
                mdot<T>(c, K, K.V, K.ld, j + 1, K.w, K.h2);
                maxpy<T>(c, n, K.V, K.ld, j + 1, K.h2, -1.0, K.w);
                mdot<T>(c, K, K.w, K.ld, 1, K.w, K.nrm, K.givens(j));
            }
            timed(c, "arnoldi/scale", 2.0 * n * sizeof(T),
                  [&] { scale_inv<T>(c, K.V + (size_t)(j + 1) * K.ld, K.w, &K.st->beta, n); });
            read_state(c, K.st);
            require(!c->hst->nan, NBP_ERR_NAN, "gmres: NaN/Inf in the Arnoldi process");
            res = c->hst->res;
            ++R.its;
            jend = j + 1;
            if (res <= tol || c->hst->beta == 0.0) break;
        }
        c->prof.launches += 1;
        k_trisolve<<<1, 1, 0, s>>>(K.H, K.m, K.g, K.y, jend);   // H is laid out with the allocated restart length
        NBP_LAUNCHED();
        maxpy<T>(c, n, K.Z, K.ld, jend, K.y, 1.0, x);
        const bool est_conv = res <= tol;
        if (est_conv && !check_true) { R.conv = 1; break; }
        // true residual: confirmation, or the next restart vector
        op(x, K.w);
        c->prof.launches++;
        k_sub<T><<<grid_for(n), 256, 0, s>>>(K.r, b, K.w, n);
        NBP_LAUNCHED();
        mdot<T>(c, K, K.r, n, 1, K.r, K.nrm);
        c->prof.launches++;
        k_gm_init<<<1, 256, 0, s>>>(K.g, m + 1, K.nrm, K.beta, K.st);
        NBP_LAUNCHED();
        read_state(c, K.st);
        res = c->hst->res;
        R.rel_true = bnorm > 0 ? res / bnorm : 0.0;
        if (res <= tol) { R.conv = 1; break; }
        if (res == 0.0) break;
        r0 = K.r;
    }
    R.rel = bnorm > 0 ? res / bnorm : 0.0;
    return R;
}

// ----------------------------------------------------------- AMG V-cycle
template <typename T> static T *wvec(Level &L, int q);
template <> double *wvec<double>(Level &L, int q) { return L.w64[q]; }
template <> float *wvec<float>(Level &L, int q) { return L.w32[q]; }
template <typename T> static const T *cinv_of(const Hier &H);
template <> const double *cinv_of<double>(const Hier &H) { return H.cinv; }
template <> const float *cinv_of<float>(const Hier &H) { return H.cinv32; }
template <typename T> static const T *dinv_of(const Level &L);
template <> const double *dinv_of<double>(const Level &L) { return L.dinv; }
template <> const float *dinv_of<float>(const Level &L) { return L.dinv32; }

struct Cheb { double theta, delta, sigma; };
static Cheb cheb_of(const Level &L) {
    const double lmax = L.rho, lmin = L.rho / L.cheb_lo;
    Cheb ch;
    ch.theta = 0.5 * (lmax + lmin);
    ch.delta = 0.5 * (lmax - lmin);
    ch.sigma = ch.theta / ch.delta;
    return ch;
}

// One Chebyshev step on level L: r = b - A x; d = c1 d + c2 Dinv r; xout = x + d
template <typename T>
static void cheb_step(nbp_ctx *c, Level &L, int vsel, const T *b, const T *x, T *xout, T *d, double c1, double c2) {
    SpmvArgs a = sargs(x, nullptr);
    a.b = b; a.dinv = dinv_of<T>(L); a.d = d; a.xout = xout; a.c1 = c1; a.c2 = c2;
    a.c1f = (float)c1; a.c2f = (float)c2;
    do_spmv<T>(c, L.M, vsel, a, EPI_CHEB, false, (&L == &c->HA.L[0]) ? CAT_CHEB_A0 : CAT_SPMV);
}

// Chebyshev smoothing of degree k on level L; from x = 0 when zero_start.
// Returns the buffer holding the result (x or alt).
// first_done: the first step from zero (d = x = Dinv b / theta) was already
// made by the restriction that produced b.
template <typename T>
static T *chebyshev(nbp_ctx *c, Level &L, int vsel, int k, const T *b, T *x, T *alt, bool zero_start,
                    bool first_done = false) {
    const int bs = L.M.br;
    const Cheb ch = cheb_of(L);
    T *d = wvec<T>(L, 4);
    double rho_old = 1.0 / ch.sigma;
    T *cur = x, *nxt = alt;
    if (k <= 0) return cur;
    if (zero_start && first_done) {
        // d and x already hold the first step
    } else if (zero_start) {
        timed(c, "amg/cheb_first", (double)L.M.nbr * bs * (bs + 3) * sizeof(T), [&] {
            k_cheb_first<T><<<grid_exact((long long)L.M.nbr * bs), 256, 0, c->s>>>(L.M.nbr, bs, dinv_of<T>(L), b,
                                                                                   (T)(1.0 / ch.theta), d, cur, nullptr);
        });
    } else {
        cheb_step<T>(c, L, vsel, b, cur, nxt, d, 0.0, 1.0 / ch.theta);
        std::swap(cur, nxt);
    }
    for (int it = 1; it < k; ++it) {
        const double rho_new = 1.0 / (2.0 * ch.sigma - rho_old);
        cheb_step<T>(c, L, vsel, b, cur, nxt, d, rho_new * rho_old, 2.0 * rho_new / ch.delta);
        std::swap(cur, nxt);
        rho_old = rho_new;
    }
    return cur;
}

template <typename T>
static void vcycle_level(nbp_ctx *c, Hier &H, int l, int vsel, const T *b, T *out, bool first_done = false);

// K-cycle on coarse level cl (Notay's Krylov-accelerated multigrid): two GCR
// steps on L_cl e = b, each preconditioned by one cycle on level cl; every
// coefficient stays on the device, so the whole cycle can be replayed from a
// CUDA graph.  x = a1 z1 + a2 z2 with a1 = (w1.b)/(w1.w1), r = b - a1 w1,
// beta = (w2.w1)/(w1.w1), w2 -= beta w1, z2 -= beta z1, a2 = (w2.r)/(w2.w2).
// w = L.M z with kd[o0] = w . da and (db set) kd[o1] = w . db: one fused
// launch (k_sell_dot) where the level's tuned kernel is a scalar sliced one,
// else the product and k_kdots
template <typename T>
static void kc_product_dots(nbp_ctx *c, Level &L, int vsel, const T *z, T *w, const T *da, const T *db, int o0, int o1) {
    const long long n = (long long)L.M.nbr * L.M.br;
    if (L.kpart && spmv_dot_ok(L.M, vsel, (int)sizeof(T), L.kpart_blocks)) {
        cudaEvent_t e0;
        prof_begin(c, e0);
        DotArgs q{da, db, L.kpart, L.kdots, o0, o1};
        const double bytes = spmv_dot<T>(L.M, vsel, sargs(z, w), q, c->s);
        std::string tag;
        if (c->prof.on) {
            tag = mat_tag(c, L.M, EPI_SET);
            tag.replace(tag.find("/set/"), 5, "/setdot/");
        }
        prof_end(c, CAT_SPMV, bytes, tag);
        return;
    }
    do_spmv<T>(c, L.M, vsel, sargs(z, w), EPI_SET, false);
    // algorithmic bytes: each distinct vector the dots read, once
    const double vn = (double)n * sizeof(T);
    const double nvec = 1.0 + (da != w ? 1.0 : 0.0) + (db && db != w && db != da ? 1.0 : 0.0);
    timed(c, "kcycle/dots", nvec * vn, [&] {
        k_kdots<T><<<kKdotBlocks, 256, 0, c->s>>>(w, da, db ? w : (const T *)nullptr, db, n, L.kdots, o0, o1);
    });
}

template <typename T>
static void kcycle_level(nbp_ctx *c, Hier &H, int cl, int vsel, const T *b, T *x, bool first_done = false) {
    Level &L = H.L[cl];
    const long long n = (long long)L.M.nbr * H.bs;
    T *r = wvec<T>(L, 5), *z1 = wvec<T>(L, 6), *w1 = wvec<T>(L, 7), *z2 = wvec<T>(L, 8), *w2 = wvec<T>(L, 9);
    const unsigned g = grid_for(n);
    const double vn = (double)n * sizeof(T);   // bytes of one level vector
    if (!first_done) copy<T>(r, b, n, c->s);   // else the restriction wrote r
    vcycle_level<T>(c, H, cl, vsel, b, z1, first_done);
    kc_product_dots<T>(c, L, vsel, z1, w1, w1, r, 0, 1);   // kd[0] = w1.w1, kd[1] = w1.r
    // algorithmic bytes: each distinct vector an update reads or writes, once
    timed(c, "kcycle/update", 3.0 * vn, [&] { k_kupd1<T><<<g, 256, 0, c->s>>>(r, w1, L.kdots, n); });
    vcycle_level<T>(c, H, cl, vsel, r, z2);
    kc_product_dots<T>(c, L, vsel, z2, w2, w1, (const T *)nullptr, 3, 3);   // kd[3] = w2.w1
    // w2 -= beta w1, z2 -= beta z1, then kd[4] = w2.w2, kd[5] = w2.r
    timed(c, "kcycle/update+dots", 7.0 * vn,
          [&] { k_kupd2_dots<T><<<kKdotBlocks, 256, 0, c->s>>>(w2, z2, w1, z1, r, L.kdots, n); });
    timed(c, "kcycle/update", 3.0 * vn, [&] { k_kupd3<T><<<g, 256, 0, c->s>>>(x, z1, z2, L.kdots, n); });
}

// V(1,1)-cycle from level l with right-hand side b; result written to out.
// first_done: the first pre-smoothing step on this level was fused into the
// restriction from the level above (d and the smoothing iterate hold it).
template <typename T>
static void vcycle_level(nbp_ctx *c, Hier &H, int l, int vsel, const T *b, T *out, bool first_done) {
    Level &L = H.L[l];
    const int bs = H.bs;
    const long long n = (long long)L.M.nbr * bs;
    const int k = H.cheb;
    if (l == H.nlev - 1) {
        if (H.cinv) {
            timed(c, "amg/coarsest_gemv", ((double)H.nc * H.nc + 2.0 * H.nc) * sizeof(T),
                  [&] {
                      const T *ci = cinv_of<T>(H);
                      if constexpr (std::is_same<T, float>::value) {
                          if (H.nc % 4 == 0 && al16(ci) && al16(b))
                              k_dense_gemv_rows<float, true><<<(unsigned)H.nc, kGemvThreads, 0, c->s>>>(ci, H.nc, b, out);
                          else
                              k_dense_gemv_rows<float, false><<<(unsigned)H.nc, kGemvThreads, 0, c->s>>>(ci, H.nc, b, out);
                      } else {
                          k_dense_gemv<T><<<grid_exact((long long)H.nc * 32), 256, 0, c->s>>>(ci, H.nc, b, out);
                      }
                  });
        } else {
            T *res = chebyshev<T>(c, L, vsel, std::max(k, 1), b, out, wvec<T>(L, 2), true);  // coarsest: smoothing only
            if (res != out) copy<T>(out, res, n, c->s);
        }
        return;
    }
    // pre-smoothing from zero; start so that the odd number of ping-pong
    // swaps (2k - 1) leaves the final result in `out`
    T *alt = wvec<T>(L, 2);
    T *x = (k > 0) ? alt : out;
    T *other = (k > 0) ? out : alt;
    if (k <= 0) fill<T>(x, T(0), n, c->s);
    T *cur = chebyshev<T>(c, L, vsel, k, b, x, other, true, first_done);
    T *oth = (cur == out) ? alt : out;
    // residual and restriction
    T *r = wvec<T>(L, 3);
    do_spmv<T>(c, L.M, vsel, [&] { SpmvArgs a = sargs(cur, r); a.b = b; return a; }(), EPI_RES, false);
    Level &Lc = H.L[l + 1];
    T *bc = wvec<T>(Lc, 0), *xc = wvec<T>(Lc, 1);
    const bool kc = H.kcycle && l + 1 < H.nlev - 1 && l + 1 <= H.kdepth;
    // below a smoothed coarse level, the restriction also makes that level's
    // first smoothing step (into the buffers its cycle uses: d = w[4], the
    // iterate w[2]) and, for a K-cycle, its copy of the right-hand side (w[5])
    const bool fuse = k > 0 && l + 1 < H.nlev - 1;
    // restriction bytes: aggregate pointers and member lists, the fine
    // residual once, the coarse right-hand side written
    const double ncv = (double)Lc.M.nbr * bs * sizeof(T);
    const double rbytes = (double)(Lc.M.nbr + 1) * 4.0 + (double)L.M.nbr * 4.0 + (double)n * sizeof(T) + ncv;
    if (fuse) {
        const Cheb chc = cheb_of(Lc);
        // + the coarse block-diagonal inverse read, d and x written (+ the copy)
        const double fbytes = rbytes + (double)Lc.M.nbr * bs * bs * sizeof(T) + 2.0 * ncv + (kc ? ncv : 0.0);
        timed(c, "amg/restrict+first", fbytes, [&] {
            k_restrict_first<T><<<grid_exact((long long)Lc.M.nbr * 8), 256, 0, c->s>>>(
                L.mptr, L.mem, Lc.M.nbr, bs, r, bc, dinv_of<T>(Lc), (T)(1.0 / chc.theta), wvec<T>(Lc, 4), wvec<T>(Lc, 2),
                kc ? wvec<T>(Lc, 5) : (T *)nullptr);
        });
    } else {
        timed(c, "amg/restrict", rbytes,
              [&] { k_restrict<T><<<grid_exact((long long)Lc.M.nbr * 8), 256, 0, c->s>>>(L.mptr, L.mem, Lc.M.nbr, bs, r, bc); });
    }
    // (a prolongation fused into the coarse level's last kernel, as a scatter
    // over each aggregate's members, was slower: uncoalesced fine updates)
    if (kc) kcycle_level<T>(c, H, l + 1, vsel, bc, xc, fuse);
    else vcycle_level<T>(c, H, l + 1, vsel, bc, xc, fuse);
    // prolongation bytes: the aggregate map, the coarse correction, x read and written
    const double pbytes = (double)L.M.nbr * 4.0 + ncv + 2.0 * n * sizeof(T);
    timed(c, "amg/prolong", pbytes, [&] {
        constexpr int W = Vec16<T>::W;
        const long long threads = L.M.nbr / W + L.M.nbr % W;
        if ((bs == 3 || bs == 1) && al16(cur) && al16(L.agg)) {
            if (bs == 3) k_prolong_v<T, 3><<<grid_exact(threads), 256, 0, c->s>>>(L.agg, L.M.nbr, xc, cur);
            else k_prolong_v<T, 1><<<grid_exact(threads), 256, 0, c->s>>>(L.agg, L.M.nbr, xc, cur);
        } else {
            k_prolong<T><<<grid_exact(n), 256, 0, c->s>>>(L.agg, L.M.nbr, bs, xc, cur);
        }
    });
    T *fin = chebyshev<T>(c, L, vsel, k, b, cur, oth, false);
    if (fin != out) copy<T>(out, fin, n, c->s);
}

// In-place autotuner of the coarse-level product kernels: for every level
// below the finest, each candidate (sliced ELL with 1, 2, 4 or 8 threads per
// row, flat kernel with g/2, g, 2g lanes per row) is timed inside the AMG
// cycle from that level down, each timed cycle preceded by a write of a
// buffer larger than L2 -- in the solve the finest level's stream evicts the
// coarse levels between cycles, so the level is first met cold and then warm
// (pre-smoothing, residual, post-smoothing), as here.  Starting at the tuned
// level keeps the finer levels' work, and its run-to-run noise, out of the
// comparison.  The median of 5 timed cycles decides.  Decisions are cached
// per (hierarchy, level shape, precision) for the life of the process so that
// every context meeting the same shapes rounds the same way.
static std::mutex g_cycle_tune_mutex;
static std::map<std::tuple<int, int, long long, int, int>, int> g_cycle_tune;

template <typename T> static void autotune_cycles(nbp_ctx *c) {
    const int vsel = amg_vsel_of(c->opt.precision);
    constexpr int kSamples = 5;
    constexpr size_t kFlushBytes = 256ull << 20;   // twice the L2
    cudaEvent_t e0, e1;
    NBP_CUDA(cudaEventCreate(&e0));
    NBP_CUDA(cudaEventCreate(&e1));
    char *flush = nullptr;
    const bool prof = c->prof.on;
    c->prof.on = false;
    try {
        for (int h = 0; h < 2; ++h) {
            Hier &H = h ? c->HS : c->HA;
            const int last = H.cinv ? H.nlev - 1 : H.nlev;   // the dense coarsest level has no product
            for (int l = 1; l < last; ++l) {
                Level &L = H.L[l];
                DMat &M = L.M;
                const auto key = std::make_tuple(h, M.nbr, (long long)M.nnz, M.br, (int)sizeof(T) * 4 + vsel);
                {
                    std::lock_guard<std::mutex> lock(g_cycle_tune_mutex);
                    auto it = g_cycle_tune.find(key);
                    if (it != g_cycle_tune.end()) { M.tuned = it->second; continue; }
                }
                if (!flush) flush = dmalloc<char>(kFlushBytes, c->s);
                const long long n = (long long)M.nbr * H.bs;
                T *b = wvec<T>(L, 0), *x = wvec<T>(L, 1);
                fill<T>(b, T(1), n, c->s);
                const int g0 = choose_group(M);
                std::vector<int> cands;
                if (M.sl_ci)
                    for (int cand : {0, kSellMT + 2, kSellMT + 4, kSellMT + 8}) cands.push_back(cand);
                cands.push_back(g0);
                if (g0 > 4) cands.push_back(g0 / 2);
                if (g0 < 32) cands.push_back(g0 * 2);
                float best = 1e30f;
                int arg = cands[0];
                for (int cand : cands) {
                    M.tuned = cand;
                    vcycle_level<T>(c, H, l, vsel, b, x);   // warm up
                    float t[kSamples];
                    for (int r = 0; r < kSamples; ++r) {
                        NBP_CUDA(cudaMemsetAsync(flush, r & 0xff, kFlushBytes, c->s));
                        NBP_CUDA(cudaEventRecord(e0, c->s));
                        vcycle_level<T>(c, H, l, vsel, b, x);
                        NBP_CUDA(cudaEventRecord(e1, c->s));
                        NBP_CUDA(cudaEventSynchronize(e1));
                        NBP_CUDA(cudaEventElapsedTime(&t[r], e0, e1));
                    }
                    std::sort(t, t + kSamples);
                    if (t[kSamples / 2] < best) { best = t[kSamples / 2]; arg = cand; }
                }
                std::lock_guard<std::mutex> lock(g_cycle_tune_mutex);
                auto it = g_cycle_tune.find(key);
                if (it != g_cycle_tune.end()) arg = it->second;
                else g_cycle_tune[key] = arg;
                M.tuned = arg;
            }
        }
    } catch (...) {
        dfree(flush, c->s);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        c->prof.on = prof;
        throw;
    }
    dfree(flush, c->s);
    c->prof.on = prof;
    c->prof.launches = 0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

static void drop_graphs(nbp_ctx *c) {
    for (auto &plane : c->graphs)
        for (auto &row : plane)
            for (auto &g : row) {
                if (g.exec) cudaGraphExecDestroy(g.exec);
                g = nbp_ctx::CycleGraph();
            }
    if (c->dl_exec) cudaGraphExecDestroy(c->dl_exec);
    c->dl_exec = nullptr;
    c->dl_key.clear();
    c->graph_gen++;
}

// One AMG cycle x = M^{-1} b.  Outside profiling the whole cycle (every level,
// every smoothing step, the coarsest solve) is replayed from a CUDA graph
// captured once per hierarchy and precision on fixed level-0 buffers; b and x
// are copied in and out around the replay.
template <typename T> static void vcycle(nbp_ctx *c, Hier &H, int vsel, const T *b, T *x) {
    cudaEvent_t e0;
    const bool on = c->prof.on;
    if (on) { e0 = c->prof.get(); NBP_CUDA(cudaEventRecord(e0, c->s)); }
    if (on || !c->use_graphs) {
        vcycle_level<T>(c, H, 0, vsel, b, x);
    } else {
        Level &L0 = H.L[0];
        T *gb = wvec<T>(L0, 0), *gx = wvec<T>(L0, 1);
        const long long n = (long long)L0.M.nbr * H.bs;
        // with a smoothed level 0, the copy of b into the replay buffer and
        // the first smoothing step from zero are one kernel outside the graph
        const bool first_in = H.cheb > 0 && H.nlev > 1;
        nbp_ctx::CycleGraph &G = c->graphs[&H == &c->HS ? 1 : 0][vsel][H.cheb];
        if (G.exec && G.cheb != H.cheb) {
            cudaGraphExecDestroy(G.exec);
            G.exec = nullptr;
        }
        if (!G.exec) {
            if (!c->cap) NBP_CUDA(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
            NBP_CUDA(cudaStreamSynchronize(c->s));
            cudaStream_t saved = c->s;
            const long long k0 = c->prof.launches;
            c->s = c->cap;
            cudaGraph_t g = nullptr;
            NBP_CUDA(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
            try {
                vcycle_level<T>(c, H, 0, vsel, gb, gx, first_in);
            } catch (...) {
                cudaStreamEndCapture(c->cap, &g);
                if (g) cudaGraphDestroy(g);
                c->s = saved;
                throw;
            }
            NBP_CUDA(cudaStreamEndCapture(c->cap, &g));
            c->s = saved;
            NBP_CUDA(cudaGraphInstantiate(&G.exec, g, 0));
            NBP_CUDA(cudaGraphDestroy(g));
            G.cheb = H.cheb;
            G.kernels = c->prof.launches - k0;
            c->prof.launches = k0;
        }
        if (first_in) {
            const Cheb ch = cheb_of(L0);
            c->prof.launches++;
            k_cheb_first<T><<<grid_exact(n), 256, 0, c->s>>>(L0.M.nbr, H.bs, dinv_of<T>(L0), b, (T)(1.0 / ch.theta),
                                                             wvec<T>(L0, 4), wvec<T>(L0, 2), gb);
            NBP_LAUNCHED();
        } else {
            copy<T>(gb, b, n, c->s);
        }
        NBP_CUDA(cudaGraphLaunch(G.exec, c->s));
        copy<T>(x, gx, n, c->s);
        c->prof.launches += G.kernels;
    }
    if (on) {
        cudaEvent_t e1 = c->prof.get();
        NBP_CUDA(cudaEventRecord(e1, c->s));
        c->prof.recs.push_back({CAT_VCYCLE, c->prof.used - 2, 0.0});
    }
}

// ------------------------------------------------- nested method pieces
template <typename T> static Krylov<T> &KA(nbp_ctx *c);
template <> Krylov<double> &KA<double>(nbp_ctx *c) { return c->KA64; }
template <> Krylov<float> &KA<float>(nbp_ctx *c) { return c->KA32; }
template <typename T> static Krylov<T> &KS(nbp_ctx *c);
template <> Krylov<double> &KS<double>(nbp_ctx *c) { return c->KS64; }
template <> Krylov<float> &KS<float>(nbp_ctx *c) { return c->KS32; }
template <typename T> static Bufs<T> &BUF(nbp_ctx *c);
template <> Bufs<double> &BUF<double>(nbp_ctx *c) { return c->B64; }
template <> Bufs<float> &BUF<float>(nbp_ctx *c) { return c->B32; }

template <typename T> __global__ void k_mul(T *y, const T *x, const T *d, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) y[i] = x[i] * d[i];
}

// GMRES(m_A) + P_A on A y = s to rtol (Sec. 3.1)
template <typename T> static GmResult solve_A(nbp_ctx *c, int vsel, const T *s, T *y, double rtol) {
    const long long n = 3LL * c->N;
    auto op = [&](const T *x, T *out) { apply_A<T>(c, vsel, x, out); };
    if (c->opt.pc_A == 1) {
        const T *dinv = BUF<T>(c).dinvA;
        auto pc = [&](const T *x, T *out) {
            c->prof.launches++;
            k_mul<T><<<grid_for(n), 256, 0, c->s>>>(out, x, dinv, n);
            NBP_LAUNCHED();
        };
        return gmres<T>(c, KA<T>(c), n, op, pc, s, y, rtol, c->opt.atol, c->opt.m_A, c->opt.nmax_A, false);
    }
    const int avsel = amg_vsel_of(c->opt.precision);
    auto pc = [&](const T *x, T *out) { vcycle<T>(c, c->HA, avsel, x, out); };
    return gmres<T>(c, KA<T>(c), n, op, pc, s, y, rtol, c->opt.atol, c->opt.m_A, c->opt.nmax_A, false);
}

// Algorithm 2: y = D x_p - C A^{-1} B x_p, inner solve to delta_I
template <typename T> static void apply_S(nbp_ctx *c, int vsel, const T *xp, T *y) {
    Bufs<T> &Bf = BUF<T>(c);
    do_spmv<T>(c, c->D, vsel, sargs(xp, y), EPI_SET, false);          // line 1: x_hat = D x_p (into y)
    do_spmv<T>(c, c->B, vsel, sargs(xp, Bf.xbar), EPI_SET, false);    // line 2: x_bar = B x_p
    GmResult R;
    as_inner_solve(c, [&] { R = solve_A<T>(c, vsel_I_of(c->opt.precision), Bf.xbar, Bf.xtil, c->opt.rtol_I); });   // line 3
    c->info.I_iters += R.its;
    c->info.n_I_solves++;
    do_spmv<T>(c, c->C, vsel, sargs(Bf.xtil, y), EPI_SUB, false);     // lines 4-5: y = x_hat - C x_tilde
}

template <typename T> __global__ void k_simple_update(T *yv, const T *yh, const T *dinv, const T *t, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        yv[i] = yh[i] - dinv[i] * t[i];
}

// SIMPLE (Sec. 3.2): Algorithm 3 with steps 3-4 replaced by a GMRES(m_S)
// solve with S_hat (P_S = AMG(S_hat)) and y_v = y_hat_v - diag(A)^{-1} B y_p.
template <typename T> static void apply_simple(nbp_ctx *c, int vsel, Bufs<T> &Bf) {
    const long long N = c->N, nv = 3 * N;
    GmResult R1 = solve_A<T>(c, vsel, Bf.sv, Bf.yvh, c->opt.rtol_A);                 // step 1
    c->info.A_iters += R1.its;
    c->info.n_A_solves++;
    do_spmv<T>(c, c->C, vsel, sargs(Bf.yvh, Bf.sp), EPI_SUB, false);                // step 2
    const DMat &Sh = c->HS.L[0].M;
    auto opH = [&](const T *x, T *out) { do_spmv<T>(c, Sh, vsel, sargs(x, out), EPI_SET, false); };
    auto pcS = [&](const T *x, T *out) { vcycle<T>(c, c->HS, amg_vsel_of(c->opt.precision), x, out); };
    GmResult R3 = gmres<T>(c, KS<T>(c), N, opH, pcS, Bf.sp, Bf.yp, c->opt.rtol_S, c->opt.atol, c->opt.m_S, c->opt.nmax_S,
                           false);                                                   // step 3'
    c->info.S_iters += R3.its;
    c->info.n_S_solves++;
    do_spmv<T>(c, c->B, vsel, sargs(Bf.yp, Bf.xbar), EPI_SET, false);               // step 4'
    c->prof.launches++;
    k_simple_update<T><<<grid_for(nv), 256, 0, c->s>>>(Bf.yv, Bf.yvh, Bf.dinvA, Bf.xbar, nv);
    NBP_LAUNCHED();
}

// Algorithm 3: y = P_SCR^{-1} s (FP64 in/out; inner type T)
template <typename T> static void apply_pscr(nbp_ctx *c, const double *s, double *y) {
    const int vsel = vsel_of(c->opt.precision);
    const long long N = c->N, nv = 3 * N;
    Bufs<T> &Bf = BUF<T>(c);
    convert<T, double>(Bf.sv, s, nv, c->s);
    convert<T, double>(Bf.sp, s + nv, N, c->s);
    if (c->opt.variant == 2) {
        apply_simple<T>(c, vsel, Bf);
        convert<double, T>(y, Bf.yv, nv, c->s);
        convert<double, T>(y + nv, Bf.yp, N, c->s);
        return;
    }
    if (c->opt.variant == 0) {
        GmResult R1 = solve_A<T>(c, vsel, Bf.sv, Bf.yvh, c->opt.rtol_A);             // step 1
        c->info.A_iters += R1.its;
        c->info.n_A_solves++;
        do_spmv<T>(c, c->C, vsel, sargs(Bf.yvh, Bf.sp), EPI_SUB, false);            // step 2: s_p -= C y_hat
    }
    auto opS = [&](const T *x, T *out) { apply_S<T>(c, vsel, x, out); };
    GmResult R3;
    if (c->opt.pc_S == 0) {
        auto pcS = [&](const T *x, T *out) { vcycle<T>(c, c->HS, amg_vsel_of(c->opt.precision), x, out); };
        R3 = gmres<T>(c, KS<T>(c), N, opS, pcS, Bf.sp, Bf.yp, c->opt.rtol_S, c->opt.atol, c->opt.m_S, c->opt.nmax_S, false);
    } else {
        auto pcI = [&](const T *x, T *out) { copy<T>(out, x, N, c->s); };
        R3 = gmres<T>(c, KS<T>(c), N, opS, pcI, Bf.sp, Bf.yp, c->opt.rtol_S, c->opt.atol, c->opt.m_S, c->opt.nmax_S, false);
    }
    c->info.S_iters += R3.its;                                                         // step 3
    c->info.n_S_solves++;
    do_spmv<T>(c, c->B, vsel, sargs(Bf.yp, Bf.sv), EPI_SUB, false);                   // step 4: s_v -= B y_p
    GmResult R5 = solve_A<T>(c, vsel, Bf.sv, Bf.yv, c->opt.rtol_A);                   // step 5
    c->info.A_iters += R5.its;
    c->info.n_A_solves++;
    convert<double, T>(y, Bf.yv, nv, c->s);
    convert<double, T>(y + nv, Bf.yp, N, c->s);
}

// y = [[A, B], [C, D]] x in FP64
static void apply_full(nbp_ctx *c, const double *x, double *y) {
    const long long nv = 3LL * c->N;
    apply_A<double>(c, 0, x, y);
    do_spmv<double>(c, c->B, 0, sargs(x + nv, y), EPI_ADD, false);
    do_spmv<double>(c, c->C, 0, sargs(x, y + nv), EPI_SET, false);
    do_spmv<double>(c, c->D, 0, sargs(x + nv, y + nv), EPI_ADD, false);
}

static void prepare_inner(nbp_ctx *c) {
    require(c->setup_done, NBP_ERR_STATE, "nbp: call nbp_setup before solving");
    require(build_level(c->opt.precision) <= build_level(c->setup_precision) || c->opt.precision == 0, NBP_ERR_STATE,
            "nbp: precision mode needs nbp_setup with that mode");
    const long long N = c->N;
    if (c->opt.precision == 0) {
        c->B64.ensure(N, c->s);
        c->prof.launches++;
        k_recip<<<grid_exact(3 * N), 256, 0, c->s>>>(3 * N, c->diagA, c->B64.dinvA);
        NBP_LAUNCHED();
    } else {
        c->B32.ensure(N, c->s);
        c->B64.ensure(N, c->s);
        c->prof.launches += 2;
        k_recip<<<grid_exact(3 * N), 256, 0, c->s>>>(3 * N, c->diagA, c->B64.dinvA);
        k_convert<float, double><<<grid_for(3 * N), 256, 0, c->s>>>(c->B32.dinvA, c->B64.dinvA, 3 * N);
        NBP_LAUNCHED();
    }
}

static void pscr(nbp_ctx *c, const double *s, double *y) {
    if (c->opt.precision == 0) apply_pscr<double>(c, s, y);
    else apply_pscr<float>(c, s, y);
}

// Outer FGMRES(m) + P_SCR (Sec. 3)
static nbp_status nested_solve(nbp_ctx *c, const double *b, double *x) {
    prepare_inner(c);
    const long long n = 4LL * c->N;
    if (!c->full_w) c->full_w = dmalloc<double>(n, c->s);
    auto op = [&](const double *xx, double *yy) { apply_full(c, xx, yy); };
    auto pc = [&](const double *ss, double *yy) { pscr(c, ss, yy); };
    GmResult R = gmres<double>(c, c->Kout, n, op, pc, b, x, c->opt.rtol, c->opt.atol, c->opt.m, c->opt.nmax, true);
    c->info.outer_iters = R.its;
    c->info.rel_res_est = R.rel;
    c->info.rel_res_true = R.rel_true;
    c->info.status = R.conv ? NBP_OK : NBP_NOT_CONVERGED;
    return R.conv ? NBP_OK : NBP_NOT_CONVERGED;
}

// ------------------------------------------------- device-driven solve
// The whole nested solve captured once as a CUDA graph in which every GMRES
// level's loop is a graph WHILE node (nested: restart cycles of the outer
// FGMRES > its iterations > the A- and S-solves of Algorithm 3 > the inner
// A-solve of Algorithm 2).  The loop state lives on the device (GmDev) and
// each iteration ends with a one-thread kernel that applies the host loop's
// stopping rule and sets the node's condition, so a solve needs no host
// round trip per iteration and many solves can run as one launch.  The
// kernels are those of the host-driven loop; the ones that depend on the
// iteration index read it from the device state.  The inner levels run one
// cycle (m >= n_max), the outer one restarts on the device.

constexpr int kDlDepth = 4;   // nesting depth of WHILE bodies

static cudaGraph_t capture_graph_of(cudaStream_t s) {
    cudaStreamCaptureStatus st;
    cudaGraph_t g = nullptr;
    NBP_CUDA(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, nullptr, nullptr, nullptr));
    require(st == cudaStreamCaptureStatusActive && g, NBP_ERR_STATE, "device loop: stream is not capturing");
    return g;
}
static cudaGraphConditionalHandle new_handle(nbp_ctx *c) {
    cudaGraphConditionalHandle h;
    NBP_CUDA(cudaGraphConditionalHandleCreate(&h, capture_graph_of(c->s), 0, 0));
    return h;
}
// kernel nodes directly in graph g (not inside its conditional nodes' bodies)
static long long kernel_nodes(cudaGraph_t g) {
    size_t n = 0;
    NBP_CUDA(cudaGraphGetNodes(g, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    if (n) NBP_CUDA(cudaGraphGetNodes(g, nodes.data(), &n));
    long long k = 0;
    for (size_t i = 0; i < n; ++i) {
        cudaGraphNodeType t;
        NBP_CUDA(cudaGraphNodeGetType(nodes[i], &t));
        if (t == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

// A WHILE node on handle h at the current capture position; body() is
// captured into its body graph on the capture stream of nesting depth
// `depth`.  Returns the kernel nodes of the body (nested bodies excluded).
template <class F> static long long emit_while(nbp_ctx *c, cudaGraphConditionalHandle h, int depth, F body) {
    require(depth < kDlDepth, NBP_ERR_STATE, "device loop: nesting too deep");
    cudaStreamCaptureStatus st;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    NBP_CUDA(cudaStreamGetCaptureInfo(c->s, &st, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    NBP_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, nd, &p));
    NBP_CUDA(cudaStreamUpdateCaptureDependencies(c->s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaGraph_t bg = p.conditional.phGraph_out[0];
    if (!c->dl_cap[depth]) NBP_CUDA(cudaStreamCreateWithFlags(&c->dl_cap[depth], cudaStreamNonBlocking));
    cudaStream_t saved = c->s;
    NBP_CUDA(cudaStreamBeginCaptureToGraph(c->dl_cap[depth], bg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    c->s = c->dl_cap[depth];
    try {
        body();
    } catch (...) {
        cudaGraph_t x = nullptr;
        cudaStreamEndCapture(c->dl_cap[depth], &x);
        c->s = saved;
        throw;
    }
    cudaGraph_t out = nullptr;
    NBP_CUDA(cudaStreamEndCapture(c->dl_cap[depth], &out));
    c->s = saved;
    return kernel_nodes(bg);
}

// The Arnoldi step of iteration st->j (the host loop's kernels, index read
// on the device): h1 = V^T w; w -= V h1, h2 = V^T w; w -= V h2, ||w|| and the
// Givens update of column j; V(:, j+1) = w / ||w||.
// One Arnoldi step of a device-driven loop, ending the iteration (its last
// kernel advances the loop state and sets the WHILE condition h)
template <typename T> static void arnoldi_dl(nbp_ctx *c, Krylov<T> &K, GmDev *st, cudaGraphConditionalHandle h) {
    const bool vec = al16(K.V) && al16(K.w) && (K.ld * (long long)sizeof(T)) % 16 == 0;
    const int *jp = &st->j;
    GivensArgs gv = K.givens(0);
    gv.jp = jp;
    if (c->gs_one_pass) gv.h2 = nullptr;
    // one pass: the multi-dot, then subtract + norm + Givens update
    const double *coef = c->gs_one_pass ? K.h1 : K.h2;
    if (vec) {
        const unsigned g1 = K.grid_md ? K.grid_md : arnoldi_grids<T>().mdot_dl_v;
        const unsigned g2 = K.grid ? K.grid : arnoldi_grids<T>().mpd_dl_v;
        k_mdot_dl<T, 8, true><<<g1, 256, 0, c->s>>>(K.V, K.ld, jp, 1, K.w, K.n, K.partial, K.h1, K.ticket, GivensArgs());
        if (!c->gs_one_pass)
            k_maxpy_dot_dl<T, kFusedCols, true><<<g2, 256, 0, c->s>>>(K.V, K.ld, jp, 1, K.h1, K.w, K.n, 0, K.partial,
                                                                      K.h2, K.ticket, GivensArgs());
        k_maxpy_dot_dl<T, kFusedCols, true><<<g2, 256, 0, c->s>>>(K.V, K.ld, jp, 1, coef, K.w, K.n, 1, K.partial, K.nrm,
                                                                  K.ticket, gv);
        k_scale_step_dl<T, true><<<grid_for(K.n / Vec16<T>::W + 1), 256, 0, c->s>>>(K.V, K.ld, st, K.w, K.st, K.n,
                                                                                   K.ticket, h);
    } else {
        const unsigned g1 = K.grid_md ? K.grid_md : arnoldi_grids<T>().mdot_dl_s;
        const unsigned g2 = K.grid ? K.grid : arnoldi_grids<T>().mpd_dl_s;
        k_mdot_dl<T, 8, false><<<g1, 256, 0, c->s>>>(K.V, K.ld, jp, 1, K.w, K.n, K.partial, K.h1, K.ticket, GivensArgs());
        if (!c->gs_one_pass)
            k_maxpy_dot_dl<T, kFusedCols, false><<<g2, 256, 0, c->s>>>(K.V, K.ld, jp, 1, K.h1, K.w, K.n, 0, K.partial,
                                                                       K.h2, K.ticket, GivensArgs());
        k_maxpy_dot_dl<T, kFusedCols, false><<<g2, 256, 0, c->s>>>(K.V, K.ld, jp, 1, coef, K.w, K.n, 1, K.partial,
                                                                   K.nrm, K.ticket, gv);
        k_scale_step_dl<T, false><<<grid_for(K.n + 1), 256, 0, c->s>>>(K.V, K.ld, st, K.w, K.st, K.n, K.ticket, h);
    }
    NBP_LAUNCHED();
}

// x += Z(:, 0..j-1) y after the cycle (j read on the device)
template <typename T> static void update_dl(nbp_ctx *c, Krylov<T> &K, GmDev *st, T *x) {
    const bool vec = al16(K.Z) && al16(x) && (K.ld * (long long)sizeof(T)) % 16 == 0;
    const unsigned grid = grid_for(K.n / (vec ? Vec16<T>::W : 1) + 1, 256, 8LL * kSMs * 4);
    if (vec) k_maxpy_dl<T, true><<<grid, 256, 0, c->s>>>(K.Z, K.ld, &st->j, 0, K.y, 1.0, x, K.n);
    else k_maxpy_dl<T, false><<<grid, 256, 0, c->s>>>(K.Z, K.ld, &st->j, 0, K.y, 1.0, x, K.n);
    NBP_LAUNCHED();
}

// One single-cycle GMRES level (inner A- and S-solves): pc(vbase, ld, jp)
// preconditions basis column j into a fixed buffer it returns; op(z, w).
template <typename T, typename Op, typename Pc>
static long long gmres_dl(nbp_ctx *c, Krylov<T> &K, long long n, GmDev *st, const double *rtol, const int *m,
                          const int *nmax, long long *its_total, long long *solves, const T *b, T *x, Pc pc, Op op,
                          int depth) {
    fill<T>(x, T(0), n, c->s);
    mdot<T>(c, K, b, n, 1, b, K.nrm);
    const cudaGraphConditionalHandle h = new_handle(c);
    k_dl_init<<<1, 256, 0, c->s>>>(st, K.g, K.m + 1, K.nrm, K.beta, K.st, rtol, &c->dl_par->atol, m, nmax, h);
    NBP_LAUNCHED();
    scale_inv<T>(c, K.V, b, K.beta, n);
    NBP_LAUNCHED();
    const long long kb = emit_while(c, h, depth, [&] {
        T *z = pc(K.V, K.ld, &st->j);
        op(z, K.w);
        k_col_put<T, T><<<grid_for(n), 256, 0, c->s>>>(K.Z, K.ld, &st->j, 0, 0, z, n);
        NBP_LAUNCHED();
        arnoldi_dl<T>(c, K, st, h);
    });
    k_dl_end<<<1, 1, 0, c->s>>>(st, K.H, K.m, K.g, K.y, its_total, solves);
    NBP_LAUNCHED();
    update_dl<T>(c, K, st, x);
    return kb;
}

// An AMG cycle on hierarchy H from basis column *jp into the hierarchy's
// level-0 output buffer (the copy-in fused with the first smoothing step, as
// the replayed cycle does); returns that buffer.
template <typename T> static T *cycle_from_col(nbp_ctx *c, Hier &H, const T *vbase, long long ld, const int *jp) {
    const int avsel = amg_vsel_of(c->opt.precision);
    Level &L0 = H.L[0];
    const long long n = (long long)L0.M.nbr * H.bs;
    T *gb = wvec<T>(L0, 0), *gx = wvec<T>(L0, 1);
    const bool first_in = H.cheb > 0 && H.nlev > 1;
    if (first_in) {
        const Cheb ch = cheb_of(L0);
        k_cheb_first_col<T><<<grid_exact(n), 256, 0, c->s>>>(L0.M.nbr, H.bs, dinv_of<T>(L0), vbase, ld, jp,
                                                             (T)(1.0 / ch.theta), wvec<T>(L0, 4), wvec<T>(L0, 2), gb);
    } else {
        k_col_get<T, T><<<grid_for(n), 256, 0, c->s>>>(gb, vbase, ld, jp, 0, 0, n);
    }
    NBP_LAUNCHED();
    vcycle_level<T>(c, H, 0, avsel, gb, gx, first_in);
    return gx;
}

// A-solve (GMRES(m_A) + P_A) of s into y inside the graph
template <typename T>
static void solve_A_dl(nbp_ctx *c, int vsel, const T *s, T *y, const double *rtol, long long *its, long long *solves,
                       int depth) {
    const long long n = 3LL * c->N;
    auto op = [&](const T *x, T *out) { apply_A<T>(c, vsel, x, out); };
    auto pc = [&](T *vbase, long long ld, const int *jp) -> T * {
        if (c->opt.pc_A == 1) {
            T *z = (T *)c->dl_zA;
            k_mul_col<T><<<grid_for(n), 256, 0, c->s>>>(z, vbase, ld, jp, BUF<T>(c).dinvA, n);
            NBP_LAUNCHED();
            return z;
        }
        return cycle_from_col<T>(c, c->HA, vbase, ld, jp);
    };
    c->dl_k_A = gmres_dl<T>(c, KA<T>(c), n, &c->dl_st[2], rtol, &c->dl_par->m_A, &c->dl_par->nmax_A, its, solves, s, y, pc,
                            op, depth);
}

// Algorithm 3 on outer basis column *jp (FP64) into c->dl_zo (FP64)
template <typename T> static double *pscr_dl(nbp_ctx *c, const double *vbase, long long ld, const int *jp, int depth) {
    const int vsel = vsel_of(c->opt.precision);
    const long long N = c->N, nv = 3 * N;
    Bufs<T> &Bf = BUF<T>(c);
    DlCounters *cnt = c->dl_cnt;
    DlParams *par = c->dl_par;
    k_col_get<T, double><<<grid_for(nv), 256, 0, c->s>>>(Bf.sv, vbase, ld, jp, 0, 0, nv);
    k_col_get<T, double><<<grid_for(N), 256, 0, c->s>>>(Bf.sp, vbase, ld, jp, 0, nv, N);
    NBP_LAUNCHED();
    if (c->opt.variant == 0) {
        solve_A_dl<T>(c, vsel, Bf.sv, Bf.yvh, &par->rtol_A, &cnt->A, &cnt->nA, depth);            // step 1
        do_spmv<T>(c, c->C, vsel, sargs(Bf.yvh, Bf.sp), EPI_SUB, false);                          // step 2
    }
    auto opS = [&](const T *x, T *out) {                                                          // Algorithm 2
        do_spmv<T>(c, c->D, vsel, sargs(x, out), EPI_SET, false);
        do_spmv<T>(c, c->B, vsel, sargs(x, Bf.xbar), EPI_SET, false);
        as_inner_solve(c, [&] {
            solve_A_dl<T>(c, vsel_I_of(c->opt.precision), Bf.xbar, Bf.xtil, &par->rtol_I, &cnt->I, &cnt->nI, depth + 1);
        });
        do_spmv<T>(c, c->C, vsel, sargs(Bf.xtil, out), EPI_SUB, false);
    };
    auto pcS = [&](T *vb, long long l, const int *j) -> T * {
        if (c->opt.pc_S == 1) {
            T *z = (T *)c->dl_zS;
            k_col_get<T, T><<<grid_for(N), 256, 0, c->s>>>(z, vb, l, j, 0, 0, N);
            NBP_LAUNCHED();
            return z;
        }
        return cycle_from_col<T>(c, c->HS, vb, l, j);
    };
    c->dl_k_S = gmres_dl<T>(c, KS<T>(c), N, &c->dl_st[1], &par->rtol_S, &par->m_S, &par->nmax_S, &cnt->S, &cnt->nS,
                            Bf.sp, Bf.yp, pcS, opS, depth);                                         // step 3
    do_spmv<T>(c, c->B, vsel, sargs(Bf.yp, Bf.sv), EPI_SUB, false);                               // step 4
    solve_A_dl<T>(c, vsel, Bf.sv, Bf.yv, &par->rtol_A, &cnt->A, &cnt->nA, depth);                // step 5
    convert<double, T>(c->dl_zo, Bf.yv, nv, c->s);
    convert<double, T>(c->dl_zo + nv, Bf.yp, N, c->s);
    return c->dl_zo;
}

// The outer FGMRES(m) with P_SCR and the true-residual check, on dl_b into dl_x
static void outer_dl(nbp_ctx *c) {
    Krylov<double> &K = c->Kout;
    const long long n = 4LL * c->N;
    GmDev *st = &c->dl_st[0];
    DlParams *par = c->dl_par;
    const double *b = c->dl_b;
    double *x = c->dl_x;
    fill<double>(x, 0.0, n, c->s);
    copy<double>(K.r, b, n, c->s);
    mdot<double>(c, K, b, n, 1, b, K.nrm);
    const cudaGraphConditionalHandle hr = new_handle(c);
    k_dl_init<<<1, 256, 0, c->s>>>(st, K.g, K.m + 1, K.nrm, K.beta, K.st, &par->rtol, &par->atol, &par->m, &par->nmax, hr);
    NBP_LAUNCHED();
    c->dl_k_cycle = emit_while(c, hr, 0, [&] {       // restart cycles
        const cudaGraphConditionalHandle hi = new_handle(c);
        k_dl_cycle_start<<<1, 1, 0, c->s>>>(st, hi);
        NBP_LAUNCHED();
        scale_inv<double>(c, K.V, K.r, K.beta, n);
        NBP_LAUNCHED();
        c->dl_k_outer = emit_while(c, hi, 1, [&] {   // iterations
            double *z = c->opt.precision == 0 ? pscr_dl<double>(c, K.V, K.ld, &st->j, 2)
                                              : pscr_dl<float>(c, K.V, K.ld, &st->j, 2);
            apply_full(c, z, K.w);
            k_col_put<double, double><<<grid_for(n), 256, 0, c->s>>>(K.Z, K.ld, &st->j, 0, 0, z, n);
            NBP_LAUNCHED();
            arnoldi_dl<double>(c, K, st, hi);
        });
        k_dl_end<<<1, 1, 0, c->s>>>(st, K.H, K.m, K.g, K.y, nullptr, nullptr);
        NBP_LAUNCHED();
        update_dl<double>(c, K, st, x);
        apply_full(c, x, K.w);                       // true residual: the next restart vector or the check
        k_sub<double><<<grid_for(n), 256, 0, c->s>>>(K.r, b, K.w, n);
        NBP_LAUNCHED();
        mdot<double>(c, K, K.r, n, 1, K.r, K.nrm);
        k_dl_restart<<<1, 256, 0, c->s>>>(st, K.nrm, K.g, K.m + 1, K.beta, K.st, hr);
        NBP_LAUNCHED();
    });
}

// Whether the device-driven solve can run with the current options: one
// cycle per inner solve (m >= n_max), not SIMPLE, not profiling.
static bool dl_supported(const nbp_ctx *c) {
    const nbp_options &o = c->opt;
    return o.m_A >= o.nmax_A && o.m_S >= o.nmax_S && o.variant != 2 && !c->prof.on;
}

// Buffers of the device-driven solve and every Krylov space at the sizes the
// options need, before any capture (a capture must not allocate).
static void dl_prepare(nbp_ctx *c) {
    prepare_inner(c);
    cudaStream_t s = c->s;
    const long long N = c->N, n = 4 * N;
    if (!c->full_w) c->full_w = dmalloc<double>(n, s);
    if (!c->dl_st) {
        c->dl_st = dmalloc<GmDev>(3, s);
        c->dl_par = dmalloc<DlParams>(1, s);
        c->dl_cnt = dmalloc<DlCounters>(1, s);
        c->dl_b = dmalloc<double>(n, s);
        c->dl_x = dmalloc<double>(n, s);
        c->dl_zo = dmalloc<double>(n, s);
        c->dl_zA = dmalloc<double>(3 * N, s);   // room for either inner type
        c->dl_zS = dmalloc<double>(N, s);
        NBP_CUDA(cudaMallocHost((void **)&c->dl_host, sizeof(GmDev)));
        NBP_CUDA(cudaMallocHost((void **)&c->dl_hcnt, sizeof(DlCounters)));
    }
    const nbp_options &o = c->opt;
    auto cl = [](int m, int nmax) { return std::max(1, std::min(m, std::max(nmax, 1))); };
    c->Kout.ensure(n, cl(o.m, o.nmax), s);
    tune_arnoldi<double>(c, c->Kout);
    if (o.precision == 0) {
        c->KA64.ensure(3 * N, cl(o.m_A, o.nmax_A), s);
        c->KS64.ensure(N, cl(o.m_S, o.nmax_S), s);
        tune_arnoldi<double>(c, c->KA64);
        tune_arnoldi<double>(c, c->KS64);
    } else {
        c->KA32.ensure(3 * N, cl(o.m_A, o.nmax_A), s);
        c->KS32.ensure(N, cl(o.m_S, o.nmax_S), s);
        tune_arnoldi<float>(c, c->KA32);
        tune_arnoldi<float>(c, c->KS32);
    }
    // the graph bakes in these buffers and option switches (the operators'
    // value copies too: a refresh of the values reallocates them)
    std::vector<const void *> key = {c->Kout.V, c->KA64.V, c->KS64.V, c->KA32.V, c->KS32.V, c->B32.sv, c->B64.sv,
                                     c->full_w, c->diagA, c->lr.lr_rp, c->lr.f,
                                     (const void *)(intptr_t)o.precision, (const void *)(intptr_t)o.variant,
                                     (const void *)(intptr_t)o.pc_A, (const void *)(intptr_t)o.pc_S,
                                     (const void *)(intptr_t)o.cheb_degree_I, (const void *)(intptr_t)o.gs_passes_I,
                                     (const void *)(intptr_t)c->Kout.m, (const void *)(intptr_t)c->KA32.m,
                                     (const void *)(intptr_t)c->KS32.m, (const void *)(intptr_t)c->KA64.m,
                                     (const void *)(intptr_t)c->KS64.m, (const void *)(intptr_t)c->Kout.grid,
                                     (const void *)(intptr_t)c->KA32.grid, (const void *)(intptr_t)c->KS32.grid,
                                     (const void *)(intptr_t)c->KA64.grid, (const void *)(intptr_t)c->KS64.grid,
                                     (const void *)(intptr_t)c->Kout.grid_md, (const void *)(intptr_t)c->KA32.grid_md,
                                     (const void *)(intptr_t)c->KS32.grid_md, (const void *)(intptr_t)c->KA64.grid_md,
                                     (const void *)(intptr_t)c->KS64.grid_md};
    for (const DMat *M : {&c->A, &c->B, &c->C, &c->D})
        for (const void *q : {(const void *)M->v, (const void *)M->v32, (const void *)M->v16, (const void *)M->sl_ptr,
                              (const void *)M->sl_ci, (const void *)M->sl_v, (const void *)M->sl_v32,
                              (const void *)M->sl2_ptr, (const void *)M->sl2_ci, (const void *)M->sl_v16})
            key.push_back(q);
    if (key != c->dl_key && c->dl_exec) {
        cudaGraphExecDestroy(c->dl_exec);
        c->dl_exec = nullptr;
    }
    c->dl_key = key;
    DlParams p;
    p.rtol = o.rtol; p.rtol_A = o.rtol_A; p.rtol_S = o.rtol_S; p.rtol_I = o.rtol_I; p.atol = o.atol;
    p.m = o.m; p.m_A = o.m_A; p.m_S = o.m_S; p.nmax = o.nmax; p.nmax_A = o.nmax_A; p.nmax_S = o.nmax_S;
    c->dl_hpar = p;
    NBP_CUDA(cudaMemcpyAsync(c->dl_par, &c->dl_hpar, sizeof(DlParams), cudaMemcpyHostToDevice, s));
    NBP_CUDA(cudaMemsetAsync(c->dl_cnt, 0, sizeof(DlCounters), s));
    // the Arnoldi kernels' grids are fixed at their first use: take them now
    (void)arnoldi_grids<float>();
    (void)arnoldi_grids<double>();
}

// Capture the device-driven solve of context c on its (capturing) stream.
static void capture_solve(nbp_ctx *c) {
    const bool prof = c->prof.on;
    c->prof.on = false;
    try {
        const long long k0 = kernel_nodes(capture_graph_of(c->s));
        outer_dl(c);
        c->dl_k_top = kernel_nodes(capture_graph_of(c->s)) - k0;
    } catch (...) {
        c->prof.on = prof;
        throw;
    }
    c->prof.on = prof;
}

static void dl_build(nbp_ctx *c) {
    if (c->dl_exec) return;
    if (!c->cap) NBP_CUDA(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
    NBP_CUDA(cudaStreamSynchronize(c->s));
    cudaStream_t saved = c->s;
    c->s = c->cap;
    cudaGraph_t g = nullptr;
    NBP_CUDA(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    try {
        capture_solve(c);
    } catch (...) {
        cudaStreamEndCapture(c->cap, &g);
        if (g) cudaGraphDestroy(g);
        c->s = saved;
        throw;
    }
    NBP_CUDA(cudaStreamEndCapture(c->cap, &g));
    c->s = saved;
    const cudaError_t e = cudaGraphInstantiate(&c->dl_exec, g, 0);
    cudaGraphDestroy(g);
    NBP_CUDA(e);
}

// Results of a finished device-driven solve (host copies taken on the stream)
static nbp_status dl_collect(nbp_ctx *c) {
    const GmDev &o = *c->dl_host;
    const DlCounters &k = *c->dl_hcnt;
    // kernels the solve ran: the captured kernel nodes times their executions
    c->prof.launches += c->dl_k_top + (long long)o.pad0 * c->dl_k_cycle + (long long)o.its * c->dl_k_outer +
                        (k.A + k.I) * c->dl_k_A + k.S * c->dl_k_S;
    require(!o.nan, NBP_ERR_NAN, "device loop: NaN/Inf in the nested solve");
    c->info.outer_iters = o.its;
    c->info.A_iters += k.A;
    c->info.S_iters += k.S;
    c->info.I_iters += k.I;
    c->info.rel_res_est = o.bnorm > 0 ? o.res / o.bnorm : 0.0;
    c->info.rel_res_true = o.rel_true;
    c->info.status = o.conv ? NBP_OK : NBP_NOT_CONVERGED;
    return o.conv ? NBP_OK : NBP_NOT_CONVERGED;
}

static void dl_fetch(nbp_ctx *c) {
    NBP_CUDA(cudaMemcpyAsync(c->dl_host, c->dl_st, sizeof(GmDev), cudaMemcpyDeviceToHost, c->s));
    NBP_CUDA(cudaMemcpyAsync(c->dl_hcnt, c->dl_cnt, sizeof(DlCounters), cudaMemcpyDeviceToHost, c->s));
}

// The nested solve as one graph launch: b in, x out (device pointers)
static nbp_status nested_solve_dl(nbp_ctx *c, const double *b, double *x) {
    dl_prepare(c);
    dl_build(c);
    const long long n = 4LL * c->N;
    copy<double>(c->dl_b, b, n, c->s);
    NBP_CUDA(cudaGraphLaunch(c->dl_exec, c->s));
    copy<double>(x, c->dl_x, n, c->s);
    dl_fetch(c);
    NBP_CUDA(cudaStreamSynchronize(c->s));
    return dl_collect(c);
}

// ---------------------------------------------------------- create / setup
__global__ void k_validate(int nbr, int nbc, const int *rp, const int *ci, long long nnz, int *bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > nbr) return;
    if (i == 0 && rp[0] != 0) atomicOr(bad, 1);
    if (i == nbr) { if ((long long)rp[nbr] != nnz) atomicOr(bad, 2); return; }
    const int a = rp[i], b = rp[i + 1];
    if (b < a) { atomicOr(bad, 4); return; }
    for (int e = a; e < b; ++e) {
        const int j = ci[e];
        if (j < 0 || j >= nbc) atomicOr(bad, 8);
        if (e > a && ci[e - 1] >= j) atomicOr(bad, 16);
    }
}
__global__ void k_finite(const double *v, long long n, int *bad) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (!isfinite(v[i])) atomicOr(bad, 32);
}

static void load_mat(nbp_ctx *c, DMat &M, const char *name, int nbr, int nbc, int br, int bc, const int32_t *rp,
                     const int32_t *ci, const double *v) {
    require(rp && ci && v, NBP_ERR_INVALID, std::string("nbp_create: null array in ") + name);
    cudaStream_t s = c->s;
    int nnz = 0;
    NBP_CUDA(cudaMemcpyAsync(&nnz, rp + nbr, sizeof(int), cudaMemcpyDeviceToHost, s));
    NBP_CUDA(cudaStreamSynchronize(s));
    require(nnz >= 0, NBP_ERR_INVALID, std::string("nbp_create: negative nnz in ") + name);
    M.nbr = nbr; M.nbc = nbc; M.br = br; M.bc = bc; M.nnz = nnz;
    M.rp = dmalloc<int>(nbr + 1, s);
    M.ci = dmalloc<int>(nnz, s);
    M.v = dmalloc<double>((long long)nnz * br * bc, s);
    NBP_CUDA(cudaMemcpyAsync(M.rp, rp, sizeof(int) * (nbr + 1), cudaMemcpyDeviceToDevice, s));
    NBP_CUDA(cudaMemcpyAsync(M.ci, ci, sizeof(int) * (size_t)nnz, cudaMemcpyDeviceToDevice, s));
    NBP_CUDA(cudaMemcpyAsync(M.v, v, sizeof(double) * (size_t)nnz * br * bc, cudaMemcpyDeviceToDevice, s));
    int *bad = dmalloc<int>(1, s);
    NBP_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    k_validate<<<grid_exact(nbr + 1), 256, 0, s>>>(nbr, nbc, M.rp, M.ci, nnz, bad);
    k_finite<<<grid_for((long long)nnz * br * bc), 256, 0, s>>>(M.v, (long long)nnz * br * bc, bad);
    NBP_LAUNCHED();
    const int b = readback(bad, s);
    dfree(bad, s);
    require(b == 0, NBP_ERR_INVALID, std::string("nbp_create: malformed ") + name + " (code " + std::to_string(b) + ")");
}

// rank-one data per velocity block row (host-side reorganisation of the small outlet arrays)
static void load_lowrank(nbp_ctx *c, const nbp_system *sys) {
    LowRank &lr = c->lr;
    cudaStream_t s = c->s;
    lr.n_out = sys->n_out;
    const int N = c->N;
    lr.lr_rp = dmalloc<int>(N + 1, s);
    if (lr.n_out <= 0) {
        lr.n_out = 0;
        NBP_CUDA(cudaMemsetAsync(lr.lr_rp, 0, sizeof(int) * (N + 1), s));
        return;
    }
    require(sys->out_ptr && sys->r, NBP_ERR_INVALID, "nbp_create: outlet arrays missing");
    std::vector<int> optr(lr.n_out + 1);
    NBP_CUDA(cudaMemcpyAsync(optr.data(), sys->out_ptr, sizeof(int) * (lr.n_out + 1), cudaMemcpyDeviceToHost, s));
    NBP_CUDA(cudaStreamSynchronize(s));
    const int no = optr[lr.n_out];
    require(optr[0] == 0 && no >= 0, NBP_ERR_INVALID, "nbp_create: bad out_ptr");
    std::vector<int> oidx(no);
    std::vector<double> oval(no);
    if (no > 0) {
        require(sys->out_idx && sys->out_val, NBP_ERR_INVALID, "nbp_create: outlet arrays missing");
        NBP_CUDA(cudaMemcpyAsync(oidx.data(), sys->out_idx, sizeof(int) * no, cudaMemcpyDeviceToHost, s));
        NBP_CUDA(cudaMemcpyAsync(oval.data(), sys->out_val, sizeof(double) * no, cudaMemcpyDeviceToHost, s));
        NBP_CUDA(cudaStreamSynchronize(s));
    }
    lr.no = no;
    lr.r_host.assign(sys->r, sys->r + lr.n_out);
    for (int k = 0; k < lr.n_out; ++k) {
        require(optr[k + 1] >= optr[k], NBP_ERR_INVALID, "nbp_create: out_ptr not monotone");
        require(std::isfinite(lr.r_host[k]), NBP_ERR_INVALID, "nbp_create: non-finite resistance weight");
    }
    std::vector<int> cnt(N + 1, 0);
    for (int q = 0; q < no; ++q) {
        require(oidx[q] >= 0 && oidx[q] < 3 * N, NBP_ERR_INVALID, "nbp_create: outlet index out of range");
        require(std::isfinite(oval[q]), NBP_ERR_INVALID, "nbp_create: non-finite outlet value");
        cnt[oidx[q] / 3 + 1]++;
    }
    for (int i = 0; i < N; ++i) cnt[i + 1] += cnt[i];
    std::vector<int> lk(no), lc(no), fillp(cnt.begin(), cnt.end() - 1);
    std::vector<double> lv(no);
    for (int k = 0; k < lr.n_out; ++k)      // k ascending inside each row
        for (int q = optr[k]; q < optr[k + 1]; ++q) {
            const int p = fillp[oidx[q] / 3]++;
            lk[p] = k; lc[p] = oidx[q] % 3; lv[p] = oval[q];
        }
    lr.optr = dmalloc<int>(lr.n_out + 1, s);
    lr.oidx = dmalloc<int>(no, s);
    lr.oval = dmalloc<double>(no, s);
    lr.r = dmalloc<double>(lr.n_out, s);
    lr.f = dmalloc<double>(lr.n_out, s);
    lr.lr_k = dmalloc<int>(no, s); lr.lr_c = dmalloc<int>(no, s); lr.lr_val = dmalloc<double>(no, s);
    NBP_CUDA(cudaMemcpyAsync(lr.optr, optr.data(), sizeof(int) * (lr.n_out + 1), cudaMemcpyHostToDevice, s));
    NBP_CUDA(cudaMemcpyAsync(lr.oidx, oidx.data(), sizeof(int) * no, cudaMemcpyHostToDevice, s));
    NBP_CUDA(cudaMemcpyAsync(lr.oval, oval.data(), sizeof(double) * no, cudaMemcpyHostToDevice, s));
    NBP_CUDA(cudaMemcpyAsync(lr.r, lr.r_host.data(), sizeof(double) * lr.n_out, cudaMemcpyHostToDevice, s));
    NBP_CUDA(cudaMemcpyAsync(lr.lr_rp, cnt.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice, s));
    NBP_CUDA(cudaMemcpyAsync(lr.lr_k, lk.data(), sizeof(int) * no, cudaMemcpyHostToDevice, s));
    NBP_CUDA(cudaMemcpyAsync(lr.lr_c, lc.data(), sizeof(int) * no, cudaMemcpyHostToDevice, s));
    NBP_CUDA(cudaMemcpyAsync(lr.lr_val, lv.data(), sizeof(double) * no, cudaMemcpyHostToDevice, s));
    NBP_CUDA(cudaStreamSynchronize(s));
}

static void free_lowrank(LowRank &lr, cudaStream_t s) {
    dfree(lr.optr, s); dfree(lr.oidx, s); dfree(lr.oval, s); dfree(lr.r, s); dfree(lr.f, s);
    dfree(lr.lr_rp, s); dfree(lr.lr_k, s); dfree(lr.lr_c, s); dfree(lr.lr_val, s);
    lr = LowRank();
}

// ------------------------------------------------ Chebyshev interval bound
// Spectral radius of the k x k matrix H (row-major) as lim ||H^m||_F^(1/m)
// (Gelfand), m = 2^40 reached by renormalised squaring, the scale carried as
// a logarithm.
static double gelfand_radius(int k, const std::vector<double> &H) {
    std::vector<double> M(H), T((size_t)k * k);
    double f = 0.0;
    for (double v : M) f += v * v;
    f = std::sqrt(f);
    if (f == 0.0) return 0.0;
    for (double &v : M) v /= f;
    double lg = std::log(f);
    const int Q = 40;
    for (int q = 0; q < Q; ++q) {
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) {
                double t = 0.0;
                for (int l = 0; l < k; ++l) t += M[(size_t)i * k + l] * M[(size_t)l * k + j];
                T[(size_t)i * k + j] = t;
            }
        double n2 = 0.0;
        for (double v : T) n2 += v * v;
        const double nn = std::sqrt(n2);
        if (nn == 0.0) return 0.0;
        for (size_t i = 0; i < T.size(); ++i) M[i] = T[i] / nn;
        lg = 2.0 * lg + std::log(nn);
    }
    return std::exp(lg / std::ldexp(1.0, Q));
}

// Upper end of level l's Chebyshev interval: min(Gershgorin bound (from
// setup), 1.1 x the spectral radius of the Hessenberg matrix of 20 Arnoldi
// steps (CGS2, FP64) on D_b^{-1} A from the normalised vector of ones).  The
// Gershgorin bound overestimates |lambda_max| 1.6-2x on these tangents, which
// weakens every smoothing step; the Ritz value approaches |lambda_max| from
// below and the factor 1.1 keeps the bound above it.  Used on AMG(A) only:
// on AMG(S_hat), smoothed with degree 1 (damped Jacobi with weight 1/theta),
// the tighter bound over-relaxes the top of the nonsymmetric spectrum and
// costs S-iterations (measured), so that hierarchy keeps Gershgorin.
constexpr int kRhoSteps = 20;
static void refine_rho(nbp_ctx *c, Hier &H, int l) {
    Level &L = H.L[l];
    if (!L.dinv) return;
    const long long n = (long long)L.M.nbr * H.bs;
    cudaStream_t s = c->s;
    Krylov<double> K;
    K.ensure(n, kRhoSteps, s);
    fill<double>(K.V, 1.0 / std::sqrt((double)n), n, s);
    std::vector<double> Hk((size_t)kRhoSteps * kRhoSteps, 0.0), h1(kRhoSteps + 1), h2(kRhoSteps + 1);
    int k = kRhoSteps;
    for (int j = 0; j < kRhoSteps; ++j) {
        do_spmv<double>(c, L.M, 0, sargs(K.V + (size_t)j * K.ld, K.w), EPI_SET, false);   // w = A v_j
        c->prof.launches++;
        k_cheb_first<double><<<grid_exact(n), 256, 0, s>>>(L.M.nbr, H.bs, L.dinv, K.w, 1.0, K.r, K.r, nullptr);
        NBP_LAUNCHED();                                                                   // r = D_b^{-1} w
        mdot<double>(c, K, K.V, K.ld, j + 1, K.r, K.h1);
        maxpy<double>(c, n, K.V, K.ld, j + 1, K.h1, -1.0, K.r);
        mdot<double>(c, K, K.V, K.ld, j + 1, K.r, K.h2);
        maxpy<double>(c, n, K.V, K.ld, j + 1, K.h2, -1.0, K.r);
        mdot<double>(c, K, K.r, K.ld, 1, K.r, K.nrm);
        double nrm2 = 0.0;
        NBP_CUDA(cudaMemcpyAsync(h1.data(), K.h1, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, s));
        NBP_CUDA(cudaMemcpyAsync(h2.data(), K.h2, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, s));
        NBP_CUDA(cudaMemcpyAsync(&nrm2, K.nrm, sizeof(double), cudaMemcpyDeviceToHost, s));
        NBP_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i <= j; ++i) Hk[(size_t)i * kRhoSteps + j] = h1[i] + h2[i];
        const double nrm = std::sqrt(std::max(nrm2, 0.0));
        if (j + 1 < kRhoSteps) Hk[(size_t)(j + 1) * kRhoSteps + j] = nrm;
        if (!(nrm > 0.0)) { k = j + 1; break; }
        if (j + 1 < kRhoSteps) {
            NBP_CUDA(cudaMemcpyAsync(K.beta, &nrm, sizeof(double), cudaMemcpyHostToDevice, s));
            scale_inv<double>(c, K.V + (size_t)(j + 1) * K.ld, K.r, K.beta, n);
            NBP_LAUNCHED();
        }
    }
    std::vector<double> Hs((size_t)k * k);
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) Hs[(size_t)i * k + j] = Hk[(size_t)i * kRhoSteps + j];
    const double est = 1.1 * gelfand_radius(k, Hs);
    NBP_CUDA(cudaStreamSynchronize(s));
    K.release(s);
    if (std::isfinite(est) && est < L.rho) L.rho = est;
}

static void refine_rhos(nbp_ctx *c, Hier &H) {
    for (int l = 0; l < H.nlev; ++l)
        if (l < H.nlev - 1 || !H.cinv) refine_rho(c, H, l);
}

// numeric: rebuild both hierarchies on the aggregates of the last full
// setup (new values, same patterns) instead of aggregating again
static void do_setup(nbp_ctx *c, bool numeric = false) {
    auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = c->s;
    drop_graphs(c);
    const int prec = build_level(c->opt.precision);
    if (!c->diagA) c->diagA = dmalloc<double>(3LL * c->N, s);
    amg_build(c->HA, c->A, c->opt, prec, s, numeric);
    refine_rhos(c, c->HA);
    build_shat(c->A, c->B, c->C, c->D, c->lr, c->N, c->Shat, c->diagA, s);
    amg_build(c->HS, c->Shat, c->opt, prec, s, numeric);   // AMG(S_hat) keeps the Gershgorin bound (see refine_rho)
    // Chebyshev intervals [rho/10, rho] on AMG(A) and [rho/3, rho] on AMG(S_hat):
    // for the degree-1 smoothing of S_hat the lower end only sets the Jacobi
    // weight (1.5 / rho); rho/3 there cut S-iterations 97 -> 91 on the 4.34M
    // tangent, while lower ends other than rho/10 were worse on A
    for (int l = 0; l < c->HA.nlev; ++l) c->HA.L[l].cheb_lo = 10.0;
    for (int l = 0; l < c->HS.nlev; ++l) c->HS.L[l].cheb_lo = 3.0;
    c->HA.kcycle = c->opt.amg_cycle == 2;
    c->HS.kcycle = c->opt.amg_cycle >= 1;
    c->HA.kdepth = c->HS.kdepth = c->opt.amg_kdepth;
    c->HA.cheb = c->opt.cheb_degree;
    c->HS.cheb = c->opt.cheb_degree_S;
    make_sell(c->A, prec, s);
    for (DMat *M : {&c->B, &c->C, &c->D}) make_sell(*M, prec, s);   // the coupling products too
    if (prec >= 1) {
        make_lowcopies(c->A, prec, s);
        make_lowcopies(c->B, prec, s);
        make_lowcopies(c->C, prec, s);
        make_lowcopies(c->D, prec, s);
    }
    // kernel choice per matrix: the fine levels use the sliced-ELL kernel;
    // coarse levels are tuned in place by timing whole AMG cycles
    c->A.tuned = c->A.sl_ci ? 0 : -1;
    for (DMat *M : {&c->B, &c->C, &c->D}) M->tuned = M->sl_ci ? 0 : -1;
    for (Hier *H : {&c->HA, &c->HS}) H->L[0].M.tuned = H->L[0].M.sl_ci ? 0 : -1;
    if (prec >= 1) autotune_cycles<float>(c);
    else autotune_cycles<double>(c);
    NBP_CUDA(cudaStreamSynchronize(s));
    c->setup_done = true;
    c->setup_precision = c->opt.precision;
    c->setup_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (c->tctx) { c->tctx->setup_done = false; }
}

static void destroy_ctx(nbp_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->dev);
    cudaStream_t s = c->s;
    if (c->tctx) destroy_ctx(c->tctx);
    drop_graphs(c);
    if (c->cap) cudaStreamDestroy(c->cap);
    for (cudaStream_t q : c->dl_cap)
        if (q) cudaStreamDestroy(q);
    dfree(c->dl_st, s); dfree(c->dl_par, s); dfree(c->dl_cnt, s); dfree(c->dl_b, s); dfree(c->dl_x, s);
    dfree(c->dl_zo, s); dfree(c->dl_zA, s); dfree(c->dl_zS, s);
    if (c->dl_host) cudaFreeHost(c->dl_host);
    if (c->dl_hcnt) cudaFreeHost(c->dl_hcnt);
    dmat_free(c->A, s); dmat_free(c->B, s); dmat_free(c->C, s); dmat_free(c->D, s); dmat_free(c->Shat, s);
    free_lowrank(c->lr, s);
    hier_free(c->HA, s); hier_free(c->HS, s);
    dfree(c->diagA, s); dfree(c->full_w, s); dfree(c->rcr_buf, s); dfree(c->rcr_bad, s);
    c->Kout.release(s); c->KA64.release(s); c->KS64.release(s); c->KA32.release(s); c->KS32.release(s);
    c->B64.release(s); c->B32.release(s);
    cudaStreamSynchronize(s);
    if (c->hst && !c->is_transposed) cudaFreeHost(c->hst);
    delete c;
}

// transposed tangent [[A^T, C^T], [B^T, D^T]] sharing the stream and outlets
static nbp_ctx *make_transposed(nbp_ctx *c) {
    nbp_ctx *t = new nbp_ctx();
    t->dev = c->dev; t->s = c->s; t->N = c->N; t->opt = c->opt; t->hst = c->hst; t->is_transposed = true;
    try {
        transpose_dmat(c->A, t->A, c->s);
        transpose_dmat(c->C, t->B, c->s);   // C^T has 3x1 blocks: plays B
        transpose_dmat(c->B, t->C, c->s);   // B^T has 1x3 blocks: plays C
        transpose_dmat(c->D, t->D, c->s);
        // same outlets and weights (the rank-one term is symmetric)
        LowRank &a = c->lr, &b = t->lr;
        b.n_out = a.n_out;
        b.r_host = a.r_host;
        const int N = c->N;
        b.lr_rp = dmalloc<int>(N + 1, c->s);
        NBP_CUDA(cudaMemcpyAsync(b.lr_rp, a.lr_rp, sizeof(int) * (N + 1), cudaMemcpyDeviceToDevice, c->s));
        if (a.n_out > 0) {
            int no = 0;
            NBP_CUDA(cudaMemcpyAsync(&no, a.optr + a.n_out, sizeof(int), cudaMemcpyDeviceToHost, c->s));
            NBP_CUDA(cudaStreamSynchronize(c->s));
            b.optr = dmalloc<int>(a.n_out + 1, c->s);
            b.oidx = dmalloc<int>(no, c->s); b.oval = dmalloc<double>(no, c->s);
            b.r = dmalloc<double>(a.n_out, c->s); b.f = dmalloc<double>(a.n_out, c->s);
            b.lr_k = dmalloc<int>(no, c->s); b.lr_c = dmalloc<int>(no, c->s); b.lr_val = dmalloc<double>(no, c->s);
            NBP_CUDA(cudaMemcpyAsync(b.optr, a.optr, sizeof(int) * (a.n_out + 1), cudaMemcpyDeviceToDevice, c->s));
            NBP_CUDA(cudaMemcpyAsync(b.oidx, a.oidx, sizeof(int) * no, cudaMemcpyDeviceToDevice, c->s));
            NBP_CUDA(cudaMemcpyAsync(b.oval, a.oval, sizeof(double) * no, cudaMemcpyDeviceToDevice, c->s));
            NBP_CUDA(cudaMemcpyAsync(b.r, a.r, sizeof(double) * a.n_out, cudaMemcpyDeviceToDevice, c->s));
            NBP_CUDA(cudaMemcpyAsync(b.lr_k, a.lr_k, sizeof(int) * no, cudaMemcpyDeviceToDevice, c->s));
            NBP_CUDA(cudaMemcpyAsync(b.lr_c, a.lr_c, sizeof(int) * no, cudaMemcpyDeviceToDevice, c->s));
            NBP_CUDA(cudaMemcpyAsync(b.lr_val, a.lr_val, sizeof(double) * no, cudaMemcpyDeviceToDevice, c->s));
        }
    } catch (...) {
        destroy_ctx(t);
        throw;
    }
    return t;
}

// dL/dr_k = -(lambda_v . a^k)(a^k . x_v): both inner products on the device
__global__ void k_adj_grad(const int *optr, const int *oidx, const double *oval, const double *lam, const double *x,
                           double *out) {
    __shared__ double r1[8], r2[8];
    const int k = blockIdx.x;
    double s1 = 0.0, s2 = 0.0;
    for (int q = optr[k] + threadIdx.x; q < optr[k + 1]; q += blockDim.x) {
        s1 += oval[q] * lam[oidx[q]];
        s2 += oval[q] * x[oidx[q]];
    }
    s1 = warp_sum(s1); s2 = warp_sum(s2);
    if ((threadIdx.x & 31) == 0) { r1[threadIdx.x >> 5] = s1; r2[threadIdx.x >> 5] = s2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += r1[w]; b += r2[w]; }
        out[k] = -a * b;
    }
}

static std::string profile_report(nbp_ctx *c);

static void finish_profile(nbp_ctx *c) {
    nbp_profile_info &p = c->pinfo;
    const double wait = p.host_wait_s;
    const long long syncs = p.host_syncs;
    p = nbp_profile_info{};
    p.host_wait_s = wait;
    p.host_syncs = syncs;
    p.kernel_launches = c->prof.launches;
    if (!c->prof.on) return;
    NBP_CUDA(cudaStreamSynchronize(c->s));
    c->report = profile_report(c);
    for (auto &r : c->prof.recs) {
        float ms = 0.f;
        NBP_CUDA(cudaEventElapsedTime(&ms, c->prof.pool[r.e0], c->prof.pool[r.e0 + 1]));
        if (r.cat == CAT_SPMV || r.cat == CAT_SPMV_A0 || r.cat == CAT_CHEB_A0) {
            p.spmv_ms += ms; p.spmv_bytes += r.bytes; p.spmv_launches++;
        }
        if (r.cat == CAT_SPMV_A0) { p.a0_ms += ms; p.a0_bytes += r.bytes; p.a0_launches++; }
        if (r.cat == CAT_CHEB_A0) { p.cheb0_ms += ms; p.cheb0_bytes += r.bytes; p.cheb0_launches++; }
        if (r.cat == CAT_ARNOLDI) { p.arnoldi_ms += ms; p.arnoldi_bytes += r.bytes; p.arnoldi_launches++; }
        if (r.cat == CAT_VCYCLE) p.vcycle_ms += ms;
    }
}

// per-tag totals of the last profiled call, as a JSON object {tag: [launches, ms, bytes]}
static std::string profile_report(nbp_ctx *c) {
    if (!c->prof.on) return "{}";
    std::map<std::string, std::tuple<long long, double, double>> m;
    for (auto &r : c->prof.recs) {
        if (r.tag.empty()) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->prof.pool[r.e0], c->prof.pool[r.e0 + 1]) != cudaSuccess) continue;
        auto &e = m[r.tag];
        std::get<0>(e) += 1;
        std::get<1>(e) += ms;
        std::get<2>(e) += r.bytes;
    }
    std::string out = "{";
    char buf[256];
    for (auto &kv : m) {
        snprintf(buf, sizeof(buf), "%s\"%s\": [%lld, %.6f, %.0f]", out.size() > 1 ? ", " : "", kv.first.c_str(),
                 std::get<0>(kv.second), std::get<1>(kv.second), std::get<2>(kv.second));
        out += buf;
    }
    return out + "}";
}

static void begin_call(nbp_ctx *c) {
    NBP_CUDA(cudaSetDevice(c->dev));
    c->prof.used = 0;
    c->prof.recs.clear();
    c->prof.launches = 0;
    c->pinfo.host_wait_s = 0.0;
    c->pinfo.host_syncs = 0;
}

}  // namespace nbp

// =================================================================== C ABI
using namespace nbp;

#define NBP_API_BEGIN(ctx) \
    if (!(ctx)) return NBP_ERR_INVALID; \
    try {
#define NBP_API_END(ctx)                                  \
    }                                                     \
    catch (const nbp::Error &e) {                         \
        (ctx)->err = e.msg;                               \
        return e.st;                                      \
    }                                                     \
    catch (const std::exception &e) {                     \
        (ctx)->err = e.what();                            \
        return NBP_ERR_CUDA;                              \
    }

extern "C" {

void nbp_default_options(nbp_options *o) {
    if (!o) return;
    o->rtol = 1e-8; o->rtol_A = 1e-3; o->rtol_S = 1e-2; o->rtol_I = 1e-2; o->atol = 1e-50;
    o->m = 200; o->m_A = 200; o->m_S = 200; o->nmax = 200; o->nmax_A = 200; o->nmax_S = 200;
    o->precision = 0; o->pc_A = 0; o->pc_S = 0; o->variant = 0;
    o->amg_max_levels = 5; o->amg_coarse_max = 300; o->cheb_degree = 2; o->theta = 0.0064;
    o->amg_cycle = 1;
    o->amg_kdepth = 2;
    o->cheb_degree_S = 1;
    o->cheb_degree_I = 1;
    o->gs_passes_I = 1;
    o->device_loop = 1;
}

static nbp_status check_options(const nbp_options *o, std::string &msg) {
    if (!(o->rtol >= 0 && o->rtol_A >= 0 && o->rtol_S >= 0 && o->rtol_I >= 0 && o->atol >= 0)) { msg = "negative tolerance"; return NBP_ERR_INVALID; }
    if (o->m < 1 || o->m_A < 1 || o->m_S < 1 || o->nmax < 1 || o->nmax_A < 1 || o->nmax_S < 1) { msg = "restart/n_max < 1"; return NBP_ERR_INVALID; }
    if (o->precision < 0 || o->precision > 4 || o->pc_A < 0 || o->pc_A > 1 || o->pc_S < 0 || o->pc_S > 1 || o->variant < 0 || o->variant > 2) { msg = "bad mode switch"; return NBP_ERR_INVALID; }
    if (o->cheb_degree < 0 || o->cheb_degree > 8 || o->cheb_degree_S < 0 || o->cheb_degree_S > 8 ||
        o->cheb_degree_I < 0 || o->cheb_degree_I > 8 || o->gs_passes_I < 1 || o->gs_passes_I > 2 || o->amg_max_levels < 1 || o->amg_cycle < 0 || o->amg_cycle > 2 || o->amg_kdepth < 1) { msg = "bad AMG option"; return NBP_ERR_INVALID; }
    if (o->device_loop < 0 || o->device_loop > 1) { msg = "device_loop must be 0 or 1"; return NBP_ERR_INVALID; }
    return NBP_OK;
}

nbp_status nbp_create(nbp_ctx **out, const nbp_system *sys, const nbp_options *opt, void *stream) {
    if (!out || !sys) return NBP_ERR_INVALID;
    *out = nullptr;
    nbp_ctx *c = new nbp_ctx();
    try {
        NBP_CUDA(cudaGetDevice(&c->dev));
        c->s = (cudaStream_t)stream;
        nbp_default_options(&c->opt);
        if (opt) c->opt = *opt;
        std::string m;
        nbp_status st = check_options(&c->opt, m);
        require(st == NBP_OK, st, "nbp_create: " + m);
        require(sys->n_nodes > 0, NBP_ERR_INVALID, "nbp_create: n_nodes must be positive");
        c->N = sys->n_nodes;
        NBP_CUDA(cudaMallocHost(&c->hst, sizeof(GmState)));
        load_mat(c, c->A, "A", c->N, c->N, 3, 3, sys->a_rowptr, sys->a_col, sys->a_val);
        load_mat(c, c->B, "B", c->N, c->N, 3, 1, sys->b_rowptr, sys->b_col, sys->b_val);
        load_mat(c, c->C, "C", c->N, c->N, 1, 3, sys->c_rowptr, sys->c_col, sys->c_val);
        load_mat(c, c->D, "D", c->N, c->N, 1, 1, sys->d_rowptr, sys->d_col, sys->d_val);
        load_lowrank(c, sys);
    } catch (const nbp::Error &e) {
        fprintf(stderr, "nbp_create: %s\n", e.msg.c_str());
        destroy_ctx(c);
        return e.st;
    } catch (const std::exception &e) {
        fprintf(stderr, "nbp_create: %s\n", e.what());
        destroy_ctx(c);
        return NBP_ERR_INVALID;
    }
    *out = c;
    return NBP_OK;
}

nbp_status nbp_setup(nbp_ctx *c) {
    NBP_API_BEGIN(c)
    begin_call(c);
    do_setup(c);
    return NBP_OK;
    NBP_API_END(c)
}

nbp_status nbp_setup_numeric(nbp_ctx *c) {
    NBP_API_BEGIN(c)
    begin_call(c);
    require(c->HA.built && c->HS.built, NBP_ERR_STATE, "nbp_setup_numeric: call nbp_setup first");
    do_setup(c, true);
    return NBP_OK;
    NBP_API_END(c)
}

nbp_status nbp_set_resistances(nbp_ctx *c, const double *r) {
    NBP_API_BEGIN(c)
    begin_call(c);
    if (c->lr.n_out == 0) return NBP_OK;
    require(r != nullptr, NBP_ERR_INVALID, "nbp_set_resistances: null r");
    for (int k = 0; k < c->lr.n_out; ++k) require(std::isfinite(r[k]), NBP_ERR_INVALID, "nbp_set_resistances: non-finite r");
    c->lr.r_host.assign(r, r + c->lr.n_out);
    NBP_CUDA(cudaMemcpyAsync(c->lr.r, c->lr.r_host.data(), sizeof(double) * c->lr.n_out, cudaMemcpyHostToDevice, c->s));
    NBP_CUDA(cudaStreamSynchronize(c->s));
    if (c->tctx) {
        c->tctx->lr.r_host = c->lr.r_host;
        NBP_CUDA(cudaMemcpyAsync(c->tctx->lr.r, c->lr.r, sizeof(double) * c->lr.n_out, cudaMemcpyDeviceToDevice, c->s));
        c->tctx->setup_done = false;
    }
    return NBP_OK;
    NBP_API_END(c)
}

nbp_status nbp_outlet_flows(nbp_ctx *c, const double *v, double *Q) {
    NBP_API_BEGIN(c)
    begin_call(c);
    require(v && (Q || c->lr.n_out == 0), NBP_ERR_INVALID, "nbp_outlet_flows: null pointer");
    launch_outlet_flows(c->lr.n_out, c->lr.optr, c->lr.oidx, c->lr.oval, v, Q, c->s);
    NBP_CUDA(cudaStreamSynchronize(c->s));
    return NBP_OK;
    NBP_API_END(c)
}

nbp_status nbp_rcr_update(nbp_ctx *c, const nbp_rcr *p, const double *v_np1, double dt, int32_t nts, double scale,
                          double *Q_np1, double *P_np1, double *Pi_np1, double *m) {
    NBP_API_BEGIN(c)
    begin_call(c);
    const int n = c->lr.n_out;
    if (n == 0) return NBP_OK;
    require(v_np1 && rcr_params_ok(p) && nts >= 1 && dt > 0.0 && std::isfinite(scale), NBP_ERR_INVALID,
            "nbp_rcr_update: bad arguments");
    if (!c->rcr_buf) {
        c->rcr_buf = dmalloc<double>(3LL * n, c->s);
        c->rcr_bad = dmalloc<int>(1, c->s);
    }
    double *Q = Q_np1 ? Q_np1 : c->rcr_buf;
    double *mk = m ? m : c->rcr_buf + n;
    double *rnew = c->rcr_buf + 2LL * n;
    NBP_CUDA(cudaMemsetAsync(c->rcr_bad, 0, sizeof(int), c->s));
    launch_outlet_flows(n, c->lr.optr, c->lr.oidx, c->lr.oval, v_np1, Q, c->s);
    launch_rcr_step(n, *p, Q, dt, nts, P_np1, Pi_np1, mk, rnew, scale, c->rcr_bad, c->s);
    int bad = 0;
    std::vector<double> r(n);
    NBP_CUDA(cudaMemcpyAsync(&bad, c->rcr_bad, sizeof(int), cudaMemcpyDeviceToHost, c->s));
    NBP_CUDA(cudaMemcpyAsync(r.data(), rnew, sizeof(double) * n, cudaMemcpyDeviceToHost, c->s));
    NBP_CUDA(cudaStreamSynchronize(c->s));
    require(!bad, NBP_ERR_NAN, "nbp_rcr_update: non-finite stiffness m^k");
    // install the weights (device copy in stream order; host copy for the transposed context)
    NBP_CUDA(cudaMemcpyAsync(c->lr.r, rnew, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->s));
    c->lr.r_host = r;
    if (c->tctx) {
        c->tctx->lr.r_host = r;
        NBP_CUDA(cudaMemcpyAsync(c->tctx->lr.r, rnew, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->s));
        c->tctx->setup_done = false;
    }
    NBP_CUDA(cudaStreamSynchronize(c->s));
    return NBP_OK;
    NBP_API_END(c)
}

static nbp_status solve_common(nbp_ctx *c, const double *b, double *x, const nbp_options *opt, nbp_info *info) {
    nbp_options saved = c->opt;
    if (opt) {
        std::string m;
        nbp_status st = check_options(opt, m);
        require(st == NBP_OK, st, "nbp_solve: " + m);
        c->opt = *opt;
    }
    memset(&c->info, 0, sizeof(c->info));
    auto t0 = std::chrono::steady_clock::now();
    nbp_status st;
    try {
        st = (c->opt.device_loop && dl_supported(c)) ? nested_solve_dl(c, b, x) : nested_solve(c, b, x);
    } catch (...) {
        c->opt = saved;
        throw;
    }
    NBP_CUDA(cudaStreamSynchronize(c->s));
    c->info.solve_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    c->info.setup_s = c->setup_s;
    c->opt = saved;
    finish_profile(c);
    if (info) *info = c->info;
    return st;
}

nbp_status nbp_solve(nbp_ctx *c, const double *b, double *x, const nbp_options *opt, nbp_info *info) {
    NBP_API_BEGIN(c)
    require(b && x, NBP_ERR_INVALID, "nbp_solve: null vector");
    begin_call(c);
    return solve_common(c, b, x, opt, info);
    NBP_API_END(c)
}

nbp_status nbp_solve_host(nbp_ctx *c, const double *bh, double *xh, const nbp_options *opt, nbp_info *info) {
    NBP_API_BEGIN(c)
    require(bh && xh, NBP_ERR_INVALID, "nbp_solve_host: null vector");
    begin_call(c);
    const long long n = 4LL * c->N;
    double *b = dmalloc<double>(n, c->s), *x = dmalloc<double>(n, c->s);
    nbp_status st;
    try {
        NBP_CUDA(cudaMemcpyAsync(b, bh, sizeof(double) * n, cudaMemcpyHostToDevice, c->s));
        st = solve_common(c, b, x, opt, info);
        NBP_CUDA(cudaMemcpyAsync(xh, x, sizeof(double) * n, cudaMemcpyDeviceToHost, c->s));
        NBP_CUDA(cudaStreamSynchronize(c->s));
    } catch (...) {
        dfree(b, c->s); dfree(x, c->s);
        throw;
    }
    dfree(b, c->s); dfree(x, c->s);
    return st;
    NBP_API_END(c)
}

nbp_status nbp_adjoint(nbp_ctx *c, const double *g, const double *x, double *lambda, double *dL_dr, nbp_info *info) {
    NBP_API_BEGIN(c)
    require(g && x && lambda, NBP_ERR_INVALID, "nbp_adjoint: null vector");
    begin_call(c);
    require(c->setup_done, NBP_ERR_STATE, "nbp_adjoint: call nbp_setup first");
    if (!c->tctx) c->tctx = make_transposed(c);
    nbp_ctx *t = c->tctx;
    t->opt = c->opt;
    if (!t->setup_done) do_setup(t);
    t->prof.on = c->prof.on;
    begin_call(t);
    nbp_status st;
    try {
        st = solve_common(t, g, lambda, nullptr, info);
    } catch (const nbp::Error &e) {
        c->err = e.msg;
        return e.st;
    }
    if (dL_dr && c->lr.n_out > 0) {
        double *d = dmalloc<double>(c->lr.n_out, c->s);
        k_adj_grad<<<c->lr.n_out, 256, 0, c->s>>>(c->lr.optr, c->lr.oidx, c->lr.oval, lambda, x, d);
        NBP_LAUNCHED();
        NBP_CUDA(cudaMemcpyAsync(dL_dr, d, sizeof(double) * c->lr.n_out, cudaMemcpyDeviceToHost, c->s));
        NBP_CUDA(cudaStreamSynchronize(c->s));
        dfree(d, c->s);
    }
    c->pinfo = t->pinfo;
    return st;
    NBP_API_END(c)
}

nbp_status nbp_destroy(nbp_ctx *c) {
    if (!c) return NBP_ERR_INVALID;
    destroy_ctx(c);
    return NBP_OK;
}

const char *nbp_last_error(const nbp_ctx *c) { return c ? c->err.c_str() : "null context"; }

nbp_status nbp_apply_A(nbp_ctx *c, const void *x, void *y, int32_t precision) {
    NBP_API_BEGIN(c)
    require(x && y, NBP_ERR_INVALID, "nbp_apply_A: null vector");
    begin_call(c);
    if (precision == 0) apply_A<double>(c, 0, (const double *)x, (double *)y);
    else {
        require(c->setup_done && build_level(c->setup_precision) >= precision, NBP_ERR_STATE, "nbp_apply_A: setup with that precision first");
        apply_A<float>(c, vsel_of(precision), (const float *)x, (float *)y);
    }
    NBP_CUDA(cudaStreamSynchronize(c->s));
    finish_profile(c);
    return NBP_OK;
    NBP_API_END(c)
}

nbp_status nbp_apply_full(nbp_ctx *c, const double *x, double *y) {
    NBP_API_BEGIN(c)
    require(x && y, NBP_ERR_INVALID, "nbp_apply_full: null vector");
    begin_call(c);
    apply_full(c, x, y);
    NBP_CUDA(cudaStreamSynchronize(c->s));
    return NBP_OK;
    NBP_API_END(c)
}

nbp_status nbp_apply_S(nbp_ctx *c, const double *xp, double *y) {
    NBP_API_BEGIN(c)
    require(xp && y, NBP_ERR_INVALID, "nbp_apply_S: null vector");
    begin_call(c);
    nbp_options saved = c->opt;
    c->opt.precision = 0;
    try { prepare_inner(c); apply_S<double>(c, 0, xp, y); } catch (...) { c->opt = saved; throw; }
    c->opt = saved;
    NBP_CUDA(cudaStreamSynchronize(c->s));
    return NBP_OK;
    NBP_API_END(c)
}

nbp_status nbp_apply_pscr(nbp_ctx *c, const double *sv, double *y) {
    NBP_API_BEGIN(c)
    require(sv && y, NBP_ERR_INVALID, "nbp_apply_pscr: null vector");
    begin_call(c);
    memset(&c->info, 0, sizeof(c->info));
    prepare_inner(c);
    pscr(c, sv, y);
    NBP_CUDA(cudaStreamSynchronize(c->s));
    return NBP_OK;
    NBP_API_END(c)
}

nbp_status nbp_solve_A(nbp_ctx *c, const double *sv, double *y, double rtol, int32_t *iters) {
    NBP_API_BEGIN(c)
    require(sv && y, NBP_ERR_INVALID, "nbp_solve_A: null vector");
    begin_call(c);
    nbp_options saved = c->opt;
    c->opt.precision = 0;
    GmResult R;
    try { prepare_inner(c); R = solve_A<double>(c, 0, sv, y, rtol); } catch (...) { c->opt = saved; throw; }
    c->opt = saved;
    if (iters) *iters = R.its;
    NBP_CUDA(cudaStreamSynchronize(c->s));
    return R.conv ? NBP_OK : NBP_NOT_CONVERGED;
    NBP_API_END(c)
}

nbp_status nbp_vcycle(nbp_ctx *c, int32_t which, const double *b, double *x) {
    NBP_API_BEGIN(c)
    require(b && x, NBP_ERR_INVALID, "nbp_vcycle: null vector");
    require(c->setup_done, NBP_ERR_STATE, "nbp_vcycle: call nbp_setup first");
    begin_call(c);
    vcycle<double>(c, which ? c->HS : c->HA, 0, b, x);
    NBP_CUDA(cudaStreamSynchronize(c->s));
    return NBP_OK;
    NBP_API_END(c)
}

int32_t nbp_amg_level_sizes(nbp_ctx *c, int32_t which, int32_t *rows, int64_t *nnz, int32_t max_levels) {
    if (!c || !c->setup_done) return 0;
    Hier &H = which ? c->HS : c->HA;
    for (int l = 0; l < H.nlev && l < max_levels; ++l) {
        if (rows) rows[l] = H.L[l].M.nbr;
        if (nnz) nnz[l] = H.L[l].M.nnz;
    }
    return H.nlev;
}

nbp_status nbp_amg_level_get(nbp_ctx *c, int32_t which, int32_t l, int32_t *rowptr, int32_t *col, double *val, int32_t *agg,
                             double *rho) {
    NBP_API_BEGIN(c)
    require(c->setup_done, NBP_ERR_STATE, "nbp_amg_level_get: call nbp_setup first");
    Hier &H = which ? c->HS : c->HA;
    require(l >= 0 && l < H.nlev, NBP_ERR_INVALID, "nbp_amg_level_get: level out of range");
    Level &L = H.L[l];
    cudaStream_t s = c->s;
    if (rowptr) NBP_CUDA(cudaMemcpyAsync(rowptr, L.M.rp, sizeof(int) * (L.M.nbr + 1), cudaMemcpyDeviceToHost, s));
    if (col) NBP_CUDA(cudaMemcpyAsync(col, L.M.ci, sizeof(int) * L.M.nnz, cudaMemcpyDeviceToHost, s));
    if (val) NBP_CUDA(cudaMemcpyAsync(val, L.M.v, sizeof(double) * L.M.nnz * L.M.bb(), cudaMemcpyDeviceToHost, s));
    if (agg && L.agg) NBP_CUDA(cudaMemcpyAsync(agg, L.agg, sizeof(int) * L.M.nbr, cudaMemcpyDeviceToHost, s));
    if (rho) *rho = L.rho;
    NBP_CUDA(cudaStreamSynchronize(s));
    return NBP_OK;
    NBP_API_END(c)
}

int64_t nbp_shat_nnz(nbp_ctx *c) { return (c && c->setup_done) ? c->Shat.nnz : -1; }

nbp_status nbp_shat_get(nbp_ctx *c, int32_t *rowptr, int32_t *col, double *val) {
    NBP_API_BEGIN(c)
    require(c->setup_done, NBP_ERR_STATE, "nbp_shat_get: call nbp_setup first");
    cudaStream_t s = c->s;
    if (rowptr) NBP_CUDA(cudaMemcpyAsync(rowptr, c->Shat.rp, sizeof(int) * (c->N + 1), cudaMemcpyDeviceToHost, s));
    if (col) NBP_CUDA(cudaMemcpyAsync(col, c->Shat.ci, sizeof(int) * c->Shat.nnz, cudaMemcpyDeviceToHost, s));
    if (val) NBP_CUDA(cudaMemcpyAsync(val, c->Shat.v, sizeof(double) * c->Shat.nnz, cudaMemcpyDeviceToHost, s));
    NBP_CUDA(cudaStreamSynchronize(s));
    return NBP_OK;
    NBP_API_END(c)
}

nbp_status nbp_profile(nbp_ctx *c, int32_t enable) {
    if (!c) return NBP_ERR_INVALID;
    c->prof.on = enable != 0;
    if (c->tctx) c->tctx->prof.on = c->prof.on;
    return NBP_OK;
}

nbp_status nbp_profile_get(nbp_ctx *c, nbp_profile_info *out) {
    if (!c || !out) return NBP_ERR_INVALID;
    *out = c->pinfo;
    return NBP_OK;
}

const char *nbp_profile_report(const nbp_ctx *c) { return c ? c->report.c_str() : "{}"; }

}  // extern "C"

// ============================================================ batched solves
// Many independent tangents solved concurrently: one context and one CUDA
// stream per instance, a pool of host threads driving the instances' nested
// solves so that their kernels (and graph replays) overlap on the GPU.
#include <atomic>
#include <thread>

struct nbp_batch {
    std::vector<nbp_ctx *> ctx;
    std::vector<cudaStream_t> streams;
    int dev = 0;
    std::string err;
    // one graph with every instance's device-driven solve as a parallel
    // branch (device_loop = 1), and what it was captured from
    cudaStream_t s0 = nullptr;
    cudaGraphExec_t dl_exec = nullptr;
    std::vector<unsigned long long> dl_gen;
    std::vector<std::vector<const void *>> dl_key;
    std::vector<cudaEvent_t> ev;
};

namespace nbp {
// Runs f(i) for every instance on a pool of host threads (one per hardware
// thread, at most one per instance).  Instances are handed out largest
// first (longest-processing-time order), so that the largest solves start
// early and the small ones fill in behind them.
template <typename F> static nbp_status batch_run(nbp_batch *B, F f) {
    const int n = (int)B->ctx.size();
    const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
    const int nt = std::max(1, std::min(n, hw));
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return B->ctx[a]->N > B->ctx[b]->N; });
    std::atomic<int> next(0);
    std::vector<nbp_status> st(n, NBP_OK);
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t)
        pool.emplace_back([&]() {
            cudaSetDevice(B->dev);
            for (int k = next++; k < n; k = next++) st[order[k]] = f(order[k]);
        });
    for (auto &th : pool) th.join();
    nbp_status worst = NBP_OK;
    for (int i = 0; i < n; ++i)
        if (st[i] != NBP_OK && (worst == NBP_OK || worst == NBP_NOT_CONVERGED)) {
            worst = st[i];
            if (st[i] != NBP_NOT_CONVERGED) B->err = "instance " + std::to_string(i) + ": " + B->ctx[i]->err;
        }
    return worst;
}
}  // namespace nbp

extern "C" {

nbp_status nbp_batch_create(nbp_batch **out, int32_t count, const nbp_system *systems, const nbp_options *opt) {
    if (!out || !systems || count <= 0) return NBP_ERR_INVALID;
    *out = nullptr;
    nbp_batch *B = new nbp_batch();
    cudaGetDevice(&B->dev);
    for (int i = 0; i < count; ++i) {
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) { nbp_batch_destroy(B); return NBP_ERR_CUDA; }
        B->streams.push_back(s);
        nbp_ctx *c = nullptr;
        nbp_status st = nbp_create(&c, &systems[i], opt, (void *)s);
        if (st != NBP_OK) { nbp_batch_destroy(B); return st; }
        B->ctx.push_back(c);
    }
    *out = B;
    return NBP_OK;
}

nbp_status nbp_batch_setup(nbp_batch *B) {
    if (!B) return NBP_ERR_INVALID;
    return nbp::batch_run(B, [&](int i) { return nbp_setup(B->ctx[i]); });
}

namespace nbp {
// Every instance's device-driven nested solve in one graph launch on B->s0:
// the right-hand sides are copied in, the graph (one parallel branch per
// instance, captured once and kept while no instance's buffers or options
// change) runs, the solutions are copied out and the counters read.
static nbp_status batch_solve_dl(nbp_batch *B, const double *const *b, double *const *x, const nbp_options *opt,
                                 nbp_info *infos) {
    const int n = (int)B->ctx.size();
    std::vector<nbp_options> saved(n);
    for (int i = 0; i < n; ++i) {
        nbp_ctx *c = B->ctx[i];
        saved[i] = c->opt;
        c->opt = *opt;
        memset(&c->info, 0, sizeof(c->info));
    }
    auto restore = [&] {
        for (int i = 0; i < n; ++i) B->ctx[i]->opt = saved[i];
    };
    try {
        if (!B->s0) NBP_CUDA(cudaStreamCreateWithFlags(&B->s0, cudaStreamNonBlocking));
        if ((int)B->ev.size() < n + 1) {
            for (int i = (int)B->ev.size(); i < n + 1; ++i) {
                cudaEvent_t e;
                NBP_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
                B->ev.push_back(e);
            }
        }
        bool stale = B->dl_exec == nullptr || (int)B->dl_gen.size() != n;
        for (int i = 0; i < n; ++i) {
            nbp_ctx *c = B->ctx[i];
            require(dl_supported(c), NBP_ERR_INVALID, "nbp_batch_solve: device_loop needs m_A >= nmax_A, m_S >= nmax_S and "
                                                      "variant 0 or 1");
            dl_prepare(c);                      // buffers, options upload, counters reset (instance stream)
            if (!stale && (B->dl_gen[i] != c->graph_gen || B->dl_key[i] != c->dl_key)) stale = true;
            NBP_CUDA(cudaEventRecord(B->ev[i], c->s));
            NBP_CUDA(cudaStreamWaitEvent(B->s0, B->ev[i], 0));
        }
        if (stale) {
            if (B->dl_exec) cudaGraphExecDestroy(B->dl_exec);
            B->dl_exec = nullptr;
            NBP_CUDA(cudaStreamSynchronize(B->s0));
            for (int i = 0; i < n; ++i) NBP_CUDA(cudaStreamSynchronize(B->ctx[i]->s));
            cudaGraph_t g = nullptr;
            NBP_CUDA(cudaStreamBeginCapture(B->s0, cudaStreamCaptureModeThreadLocal));
            try {
                // branches made largest instance first (the order the graph's
                // root nodes are issued in)
                std::vector<int> order(n);
                std::iota(order.begin(), order.end(), 0);
                std::stable_sort(order.begin(), order.end(), [&](int p, int q) { return B->ctx[p]->N > B->ctx[q]->N; });
                NBP_CUDA(cudaEventRecord(B->ev[n], B->s0));
                for (int i : order) NBP_CUDA(cudaStreamWaitEvent(B->ctx[i]->s, B->ev[n], 0));   // fork
                for (int i : order) capture_solve(B->ctx[i]);
                for (int i = 0; i < n; ++i) {                                                         // join
                    NBP_CUDA(cudaEventRecord(B->ev[i], B->ctx[i]->s));
                    NBP_CUDA(cudaStreamWaitEvent(B->s0, B->ev[i], 0));
                }
            } catch (...) {
                cudaStreamEndCapture(B->s0, &g);
                if (g) cudaGraphDestroy(g);
                throw;
            }
            NBP_CUDA(cudaStreamEndCapture(B->s0, &g));
            const cudaError_t e = cudaGraphInstantiate(&B->dl_exec, g, 0);
            cudaGraphDestroy(g);
            NBP_CUDA(e);
            B->dl_gen.assign(n, 0);
            B->dl_key.assign(n, {});
            for (int i = 0; i < n; ++i) {
                B->dl_gen[i] = B->ctx[i]->graph_gen;
                B->dl_key[i] = B->ctx[i]->dl_key;
            }
        }
        for (int i = 0; i < n; ++i) {
            nbp_ctx *c = B->ctx[i];
            NBP_CUDA(cudaMemcpyAsync(c->dl_b, b[i], sizeof(double) * 4 * c->N, cudaMemcpyDeviceToDevice, B->s0));
        }
        NBP_CUDA(cudaGraphLaunch(B->dl_exec, B->s0));
        for (int i = 0; i < n; ++i) {
            nbp_ctx *c = B->ctx[i];
            NBP_CUDA(cudaMemcpyAsync(x[i], c->dl_x, sizeof(double) * 4 * c->N, cudaMemcpyDeviceToDevice, B->s0));
            NBP_CUDA(cudaMemcpyAsync(c->dl_host, c->dl_st, sizeof(GmDev), cudaMemcpyDeviceToHost, B->s0));
            NBP_CUDA(cudaMemcpyAsync(c->dl_hcnt, c->dl_cnt, sizeof(DlCounters), cudaMemcpyDeviceToHost, B->s0));
        }
        NBP_CUDA(cudaStreamSynchronize(B->s0));
    } catch (const Error &e) {
        restore();
        B->err = e.msg;
        return e.st;
    } catch (const std::exception &e) {
        restore();
        B->err = e.what();
        return NBP_ERR_CUDA;
    }
    nbp_status worst = NBP_OK;
    for (int i = 0; i < n; ++i) {
        nbp_ctx *c = B->ctx[i];
        nbp_status st;
        try {
            st = dl_collect(c);
        } catch (const Error &e) {
            st = e.st;
            c->err = e.msg;
        }
        c->info.setup_s = c->setup_s;
        if (infos) infos[i] = c->info;
        if (st != NBP_OK && (worst == NBP_OK || worst == NBP_NOT_CONVERGED)) {
            worst = st;
            if (st != NBP_NOT_CONVERGED) B->err = "instance " + std::to_string(i) + ": " + c->err;
        }
    }
    restore();
    return worst;
}
}  // namespace nbp

nbp_status nbp_batch_solve(nbp_batch *B, const double *const *b, double *const *x, const nbp_options *opt, nbp_info *infos) {
    if (!B || !b || !x) return NBP_ERR_INVALID;
    if (opt && opt->device_loop) {
        std::string m;
        const nbp_status st = check_options(opt, m);
        if (st != NBP_OK) { B->err = "nbp_batch_solve: " + m; return st; }
        for (int i = 0; i < (int)B->ctx.size(); ++i)
            if (!B->ctx[i]->setup_done) { B->err = "nbp_batch_solve: instance " + std::to_string(i) + " not set up"; return NBP_ERR_STATE; }
        cudaSetDevice(B->dev);
        return nbp::batch_solve_dl(B, b, x, opt, infos);
    }
    return nbp::batch_run(B, [&](int i) { return nbp_solve(B->ctx[i], b[i], x[i], opt, infos ? &infos[i] : nullptr); });
}

int32_t nbp_batch_size(const nbp_batch *B) { return B ? (int32_t)B->ctx.size() : 0; }

nbp_status nbp_batch_destroy(nbp_batch *B) {
    if (!B) return NBP_ERR_INVALID;
    if (B->dl_exec) cudaGraphExecDestroy(B->dl_exec);
    for (auto e : B->ev) cudaEventDestroy(e);
    if (B->s0) {
        cudaStreamSynchronize(B->s0);
        cudaStreamDestroy(B->s0);
    }
    for (auto *c : B->ctx) nbp_destroy(c);
    for (auto s : B->streams) cudaStreamDestroy(s);
    delete B;
    return NBP_OK;
}

const char *nbp_batch_last_error(const nbp_batch *B) { return B ? B->err.c_str() : "null batch"; }

}  // extern "C"

// ============================================ VMS assembly and Newton time step
// The predictor multi-corrector of Sec. 2.5 around the nested solve: residual
// and tangent assembled on the device (vms.cu), the RCR outlet coupling on the
// device (rcr.cu), the tangent values installed in the context in place and
// the preconditioner rebuilt for every corrector (the tangent changes).
namespace nbp {

constexpr int kNormBlocks = 1024;

__global__ void k_sumsq_part(long long n, const double *x, double *part) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc += x[i] * x[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}
__global__ void k_sum_parts(int n, const double *part, double *out) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}
// predictor (Sec. 2.5): y = y_n, ydot = (gamma - 1) / gamma ydot_n
__global__ void k_newton_predict(long long n, const double *y_n, const double *yd_n, double coef, double *y, double *yd) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        y[i] = y_n[i];
        yd[i] = coef * yd_n[i];
    }
}
// intermediate stages (Sec. 2.5 step 4)
__global__ void k_newton_stage(long long n, const double *y_n, const double *yd_n, const double *y, const double *yd,
                               double af, double am, double *yaf, double *ydam) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        yaf[i] = y_n[i] + af * (y[i] - y_n[i]);
        ydam[i] = yd_n[i] + am * (yd[i] - yd_n[i]);
    }
}
// update (Sec. 2.5 step 10) with the velocity increments of Dirichlet nodes set to zero
__global__ void k_newton_update(int N, const uint8_t *dir, const double *dx, double gdt, double *y, double *yd) {
    const long long n = 4LL * N;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double d = (i < 3LL * N && dir[i / 3]) ? 0.0 : dx[i];
        yd[i] += d;
        y[i] += gdt * d;
    }
}
__global__ void k_negate(long long n, const double *x, double *y) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = -x[i];
}
// P^k_n = R_p Q_n + Pi_n + P_d (Algorithm 1's output relation at t_n)
__global__ void k_outlet_pn(int n, const double *Rp, const double *Pi, const double *Pd, const double *Q, double *Pn) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) Pn[k] = Rp[k] * Q[k] + Pi[k] + Pd[k];
}
// P^k_{n+alpha_f} = (1 - alpha_f) P^k_n + alpha_f P^k_{n+1} (Sec. 2.5 step 5)
__global__ void k_outlet_paf(int n, const double *Pn, const double *P1, double af, double *Paf) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) Paf[k] = (1.0 - af) * Pn[k] + af * P1[k];
}

// the value-derived copies of a matrix (precision copies, sliced-ELL layouts)
static void drop_value_copies(DMat &m, cudaStream_t s) {
    dfree(m.v32, s); dfree(m.v16, s);
    dfree(m.sl_ptr, s); dfree(m.sl_ci, s); dfree(m.sl_v, s); dfree(m.sl_v32, s); dfree(m.sl_v16, s);
    dfree(m.sl2_ptr, s); dfree(m.sl2_ci, s);
    m.v32 = nullptr; m.v16 = nullptr;
    m.sl_ptr = nullptr; m.sl_ci = nullptr; m.sl_v = nullptr; m.sl_v32 = nullptr; m.sl_v16 = nullptr;
    m.sl2_ptr = nullptr; m.sl2_ci = nullptr;
}

// new values of A, B, C, D are in place: everything built from them is stale
static void values_changed(nbp_ctx *c) {
    for (DMat *M : {&c->A, &c->B, &c->C, &c->D}) drop_value_copies(*M, c->s);
    drop_graphs(c);
    c->setup_done = false;
    if (c->tctx) {
        destroy_ctx(c->tctx);
        c->tctx = nullptr;
    }
}

// New values of A, B, C, D are in place but the preconditioner built from an
// earlier tangent is kept (a lagged preconditioner): only the operators'
// sliced-ELL and precision copies are rebuilt; both AMG hierarchies, S_hat,
// diag(A) and the replayed cycle graphs stay as they are.
static void refresh_operators(nbp_ctx *c) {
    const int prec = build_level(c->setup_precision);
    // the captured device-driven solve holds the old copies' addresses
    if (c->dl_exec) cudaGraphExecDestroy(c->dl_exec);
    c->dl_exec = nullptr;
    c->dl_key.clear();
    c->graph_gen++;
    for (DMat *M : {&c->A, &c->B, &c->C, &c->D}) {
        drop_value_copies(*M, c->s);
        make_sell(*M, prec, c->s);
        if (prec >= 1) make_lowcopies(*M, prec, c->s);
        M->tuned = M->sl_ci ? 0 : -1;
    }
    if (c->tctx) {   // the transposed system belongs to the old values
        destroy_ctx(c->tctx);
        c->tctx = nullptr;
    }
}

static double norm2(const double *x, long long n, double *part, cudaStream_t s) {
    k_sumsq_part<<<kNormBlocks, 256, 0, s>>>(n, x, part);
    k_sum_parts<<<1, 256, 0, s>>>(kNormBlocks, part, part + kNormBlocks);
    NBP_LAUNCHED();
    return std::sqrt(readback(part + kNormBlocks, s));
}

}  // namespace nbp

struct nbp_vms {
    nbp_ctx *ctx = nullptr;
    nbp::VmsDev m;
    nbp::VmsConst k;
    double *yaf = nullptr, *ydam = nullptr, *R = nullptr, *dx = nullptr, *rhs = nullptr;   // 4N each
    double *ob = nullptr;        // outlet scratch: Q_n, Q, P_n, P, Pi, m, r, P_af (8 n_out)
    int *bad = nullptr;
    double *part = nullptr;      // norm partials
};

#define VMS_BEGIN(v)                     \
    if (!(v) || !(v)->ctx) return NBP_ERR_INVALID; \
    nbp_ctx *c = (v)->ctx;               \
    try {
#define VMS_END NBP_API_END(c)

namespace nbp {

static void vms_free(nbp_vms *v) {
    if (!v) return;
    cudaStream_t s = v->ctx ? v->ctx->s : nullptr;
    VmsDev &m = v->m;
    for (void *p : {(void *)m.X, (void *)m.tets, (void *)m.tris, (void *)m.dir, (void *)m.n2t_ptr, (void *)m.n2t,
                    (void *)m.n2f_ptr, (void *)m.n2f, (void *)m.sl_ptr, (void *)m.sl_src, (void *)m.fl_ptr,
                    (void *)m.fl_src, (void *)m.slot_row, (void *)m.Re, (void *)m.Rf, m.Ke, m.Kf, (void *)v->yaf,
                    (void *)v->ydam, (void *)v->R, (void *)v->dx, (void *)v->rhs, (void *)v->ob, (void *)v->bad,
                    (void *)v->part})
        dfree(p, s);
    if (s) cudaStreamSynchronize(s);
    delete v;
}

template <typename T> static T *upload(const std::vector<T> &h, cudaStream_t s) {
    T *d = dmalloc<T>(h.size(), s);
    if (!h.empty()) NBP_CUDA(cudaMemcpyAsync(d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, s));
    return d;
}

// CSR of (node -> local incidences) in ascending element order: entries w e + la
static void incidence(int N, int E, int w, const int32_t *el, std::vector<int> &ptr, std::vector<int> &idx) {
    ptr.assign(N + 1, 0);
    for (long long q = 0; q < (long long)E * w; ++q) ptr[el[q] + 1]++;
    for (int A = 0; A < N; ++A) ptr[A + 1] += ptr[A];
    idx.resize((size_t)E * w);
    std::vector<int> pos(ptr.begin(), ptr.end() - 1);
    for (int e = 0; e < E; ++e)
        for (int a = 0; a < w; ++a) idx[pos[el[(size_t)e * w + a]]++] = w * e + a;
}

// CSR of (pattern slot -> element blocks), ascending element order: entries
// w^2 e + w la + lb for every local pair (la, lb) of every element
static void slot_map(int N, const std::vector<int> &rp, const std::vector<int> &ci, int E, int w, const int32_t *el,
                     std::vector<int> &ptr, std::vector<int> &src) {
    const long long nnz = rp[N];
    std::vector<int> slot((size_t)E * w * w);
    ptr.assign(nnz + 1, 0);
    for (int e = 0; e < E; ++e)
        for (int a = 0; a < w; ++a) {
            const int A = el[(size_t)e * w + a];
            for (int b = 0; b < w; ++b) {
                const int B = el[(size_t)e * w + b];
                const int *lo = ci.data() + rp[A], *hi = ci.data() + rp[A + 1];
                const int *f = std::lower_bound(lo, hi, B);
                require(f != hi && *f == B, NBP_ERR_INVALID,
                        "nbp_vms_create: an element couples two nodes absent from the solver's pattern");
                const int sl = (int)(f - ci.data());
                slot[((size_t)e * w + a) * w + b] = sl;
                ptr[sl + 1]++;
            }
        }
    for (long long q = 0; q < nnz; ++q) ptr[q + 1] += ptr[q];
    src.resize((size_t)E * w * w);
    std::vector<int> pos(ptr.begin(), ptr.end() - 1);
    for (int e = 0; e < E; ++e)
        for (int a = 0; a < w; ++a)
            for (int b = 0; b < w; ++b) src[pos[slot[((size_t)e * w + a) * w + b]]++] = w * w * e + w * a + b;
}

static void vms_buffers(nbp_vms *v) {
    if (v->yaf) return;
    nbp_ctx *c = v->ctx;
    const long long n = 4LL * c->N;
    v->yaf = dmalloc<double>(n, c->s);
    v->ydam = dmalloc<double>(n, c->s);
    v->R = dmalloc<double>(n, c->s);
    v->dx = dmalloc<double>(n, c->s);
    v->rhs = dmalloc<double>(n, c->s);
    v->ob = dmalloc<double>(8LL * std::max(c->lr.n_out, 1), c->s);
    v->bad = dmalloc<int>(1, c->s);
}

static void vms_residual_ctx(nbp_vms *v, const double *vd, const double *vel, const double *p, const double *vtau,
                             const double *P, double *R) {
    nbp_ctx *c = v->ctx;
    const LowRank &lr = c->lr;
    vms_residual(v->m, v->k, vd, vel, p, vtau, lr.n_out, lr.lr_rp, lr.lr_k, lr.lr_c, lr.lr_val, P, R, c->s);
}

}  // namespace nbp

extern "C" {

nbp_status nbp_set_values(nbp_ctx *c, const double *a_val, const double *b_val, const double *c_val,
                          const double *d_val) {
    NBP_API_BEGIN(c)
    begin_call(c);
    require(a_val && b_val && c_val && d_val, NBP_ERR_INVALID, "nbp_set_values: null array");
    const DMat *M[4] = {&c->A, &c->B, &c->C, &c->D};
    const double *src[4] = {a_val, b_val, c_val, d_val};
    int *bad = dmalloc<int>(1, c->s);
    NBP_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), c->s));
    for (int q = 0; q < 4; ++q) {
        const long long nv = M[q]->nnz * M[q]->bb();
        if (nv == 0) continue;
        k_finite<<<grid_for(nv), 256, 0, c->s>>>(src[q], nv, bad);
        NBP_LAUNCHED();
    }
    const int b = readback(bad, c->s);
    dfree(bad, c->s);
    require(b == 0, NBP_ERR_INVALID, "nbp_set_values: non-finite value");
    for (int q = 0; q < 4; ++q) {
        const long long nv = M[q]->nnz * M[q]->bb();
        if (nv) NBP_CUDA(cudaMemcpyAsync(M[q]->v, src[q], sizeof(double) * nv, cudaMemcpyDeviceToDevice, c->s));
    }
    values_changed(c);
    NBP_CUDA(cudaStreamSynchronize(c->s));
    return NBP_OK;
    NBP_API_END(c)
}

nbp_status nbp_vms_maps(int32_t n_nodes, const int32_t *rowptr, const int32_t *col, int32_t n_el, int32_t w,
                        const int32_t *el, int32_t *inc_ptr, int32_t *inc, int32_t *slot_ptr, int32_t *slot_src) {
    try {
        require(n_nodes >= 0 && n_el >= 0 && (w == 3 || w == 4) && rowptr && col && (el || n_el == 0) && inc_ptr &&
                    inc && slot_ptr && slot_src,
                NBP_ERR_INVALID, "nbp_vms_maps: bad arguments");
        for (long long q = 0; q < (long long)n_el * w; ++q)
            require(el[q] >= 0 && el[q] < n_nodes, NBP_ERR_INVALID, "nbp_vms_maps: node id out of range");
        const long long nnz = rowptr[n_nodes];
        std::vector<int> rp(rowptr, rowptr + n_nodes + 1), ci(col, col + nnz), ip, ix, sp, ss;
        incidence(n_nodes, n_el, w, el, ip, ix);
        slot_map(n_nodes, rp, ci, n_el, w, el, sp, ss);
        std::copy(ip.begin(), ip.end(), inc_ptr);
        std::copy(ix.begin(), ix.end(), inc);
        std::copy(sp.begin(), sp.end(), slot_ptr);
        std::copy(ss.begin(), ss.end(), slot_src);
        return NBP_OK;
    } catch (const nbp::Error &e) {
        return e.st;
    } catch (const std::exception &) {
        return NBP_ERR_OOM;
    }
}

nbp_status nbp_vms_create(nbp_vms **out, nbp_ctx *c, const nbp_mesh *mesh, const nbp_vms_params *par) {
    if (!out) return NBP_ERR_INVALID;
    *out = nullptr;
    NBP_API_BEGIN(c)
    begin_call(c);
    require(mesh && par, NBP_ERR_INVALID, "nbp_vms_create: null argument");
    require(mesh->n_nodes == c->N, NBP_ERR_INVALID, "nbp_vms_create: mesh and context node counts differ");
    require(mesh->n_tets >= 0 && mesh->n_tris >= 0, NBP_ERR_INVALID, "nbp_vms_create: negative element count");
    require(mesh->X && mesh->dir && (mesh->tets || mesh->n_tets == 0) && (mesh->tris || mesh->n_tris == 0),
            NBP_ERR_INVALID, "nbp_vms_create: null mesh array");
    require(par->rho > 0 && par->mu > 0 && par->dt > 0 && par->rho_inf >= 0 && par->rho_inf <= 1 && par->beta >= 0 &&
                par->CI > 0 && par->CT > 0,
            NBP_ERR_INVALID, "nbp_vms_create: bad physical parameters");
    const int N = c->N, E = mesh->n_tets, T = mesh->n_tris;
    for (long long q = 0; q < 4LL * E; ++q)
        require(mesh->tets[q] >= 0 && mesh->tets[q] < N, NBP_ERR_INVALID, "nbp_vms_create: tet node out of range");
    for (long long q = 0; q < 3LL * T; ++q)
        require(mesh->tris[q] >= 0 && mesh->tris[q] < N, NBP_ERR_INVALID, "nbp_vms_create: triangle node out of range");
    // degenerate elements (the shape-function gradients would divide by a zero
    // volume or area): |det| must exceed 1e-12 of the cube (square) of the
    // longest edge
    auto edge = [&](int a, int b, int r) { return mesh->X[3LL * b + r] - mesh->X[3LL * a + r]; };
    for (long long e = 0; e < E; ++e) {
        const int32_t *t = mesh->tets + 4 * e;
        double d[3][3], lmax = 0.0;
        for (int k = 0; k < 3; ++k)
            for (int r = 0; r < 3; ++r) d[k][r] = edge(t[0], t[k + 1], r);
        for (int a = 0; a < 4; ++a)
            for (int b = a + 1; b < 4; ++b) {
                double l2 = 0.0;
                for (int r = 0; r < 3; ++r) l2 += edge(t[a], t[b], r) * edge(t[a], t[b], r);
                lmax = std::max(lmax, std::sqrt(l2));
            }
        const double det = d[0][0] * (d[1][1] * d[2][2] - d[1][2] * d[2][1]) -
                           d[0][1] * (d[1][0] * d[2][2] - d[1][2] * d[2][0]) +
                           d[0][2] * (d[1][0] * d[2][1] - d[1][1] * d[2][0]);
        require(std::isfinite(det) && std::fabs(det) > 1e-12 * lmax * lmax * lmax, NBP_ERR_INVALID,
                "nbp_vms_create: degenerate tet " + std::to_string(e));
    }
    for (long long f = 0; f < T; ++f) {
        const int32_t *t = mesh->tris + 3 * f;
        double c[3], l2max = 0.0;
        for (int r = 0; r < 3; ++r)
            c[r] = edge(t[0], t[1], (r + 1) % 3) * edge(t[0], t[2], (r + 2) % 3) -
                   edge(t[0], t[1], (r + 2) % 3) * edge(t[0], t[2], (r + 1) % 3);
        for (int a = 0; a < 3; ++a)
            for (int b = a + 1; b < 3; ++b) {
                double l2 = 0.0;
                for (int r = 0; r < 3; ++r) l2 += edge(t[a], t[b], r) * edge(t[a], t[b], r);
                l2max = std::max(l2max, l2);
            }
        const double area2 = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        require(std::isfinite(area2) && area2 > 1e-12 * l2max, NBP_ERR_INVALID,
                "nbp_vms_create: degenerate outlet triangle " + std::to_string(f));
    }
    std::unique_ptr<nbp_vms, void (*)(nbp_vms *)> v(new nbp_vms(), vms_free);
    v->ctx = c;
    cudaStream_t s = c->s;
    // the solver's (shared) pattern on the host
    const long long nnz = c->A.nnz;
    require(c->B.nnz == nnz && c->C.nnz == nnz && c->D.nnz == nnz, NBP_ERR_INVALID,
            "nbp_vms_create: A, B, C, D must share one pattern");
    std::vector<int> rp(N + 1), ci(nnz);
    NBP_CUDA(cudaMemcpyAsync(rp.data(), c->A.rp, sizeof(int) * (N + 1), cudaMemcpyDeviceToHost, s));
    NBP_CUDA(cudaMemcpyAsync(ci.data(), c->A.ci, sizeof(int) * nnz, cudaMemcpyDeviceToHost, s));
    NBP_CUDA(cudaStreamSynchronize(s));
    std::vector<int> n2t_ptr, n2t, n2f_ptr, n2f, sl_ptr, sl_src, fl_ptr, fl_src, slot_row(nnz);
    incidence(N, E, 4, mesh->tets, n2t_ptr, n2t);
    incidence(N, T, 3, mesh->tris, n2f_ptr, n2f);
    slot_map(N, rp, ci, E, 4, mesh->tets, sl_ptr, sl_src);
    slot_map(N, rp, ci, T, 3, mesh->tris, fl_ptr, fl_src);
    for (int A = 0; A < N; ++A)
        for (int q = rp[A]; q < rp[A + 1]; ++q) slot_row[q] = A;
    VmsDev &m = v->m;
    m.N = N; m.E = E; m.T = T; m.nnz = nnz;
    m.X = upload(std::vector<double>(mesh->X, mesh->X + 3LL * N), s);
    m.tets = upload(std::vector<int>(mesh->tets, mesh->tets + 4LL * E), s);
    m.tris = upload(std::vector<int>(mesh->tris, mesh->tris + 3LL * T), s);
    m.dir = upload(std::vector<uint8_t>(mesh->dir, mesh->dir + N), s);
    m.n2t_ptr = upload(n2t_ptr, s); m.n2t = upload(n2t, s);
    m.n2f_ptr = upload(n2f_ptr, s); m.n2f = upload(n2f, s);
    m.sl_ptr = upload(sl_ptr, s); m.sl_src = upload(sl_src, s);
    m.fl_ptr = upload(fl_ptr, s); m.fl_src = upload(fl_src, s);
    m.slot_row = upload(slot_row, s);
    m.col = c->A.ci;
    m.tangent_fp32 = par->tangent_fp32 ? 1 : 0;
    const size_t tb = m.tangent_fp32 ? sizeof(float) : sizeof(double);
    m.Re = dmalloc<double>(16LL * std::max(E, 1), s);
    m.Rf = dmalloc<double>(9LL * std::max(T, 1), s);
    m.Ke = dmalloc<char>(256LL * std::max(E, 1) * tb, s);
    m.Kf = dmalloc<char>(81LL * std::max(T, 1) * tb, s);
    v->part = dmalloc<double>(kNormBlocks + 1, s);
    VmsConst &k = v->k;
    k.rho = par->rho; k.mu = par->mu; k.dt = par->dt; k.beta = par->beta; k.CI = par->CI; k.CT = par->CT;
    k.am = 0.5 * (3.0 - par->rho_inf) / (1.0 + par->rho_inf);
    k.af = 1.0 / (1.0 + par->rho_inf);
    k.gm = 1.0 / (1.0 + par->rho_inf);
    k.c = k.af * k.gm * par->dt;
    NBP_CUDA(cudaStreamSynchronize(s));
    *out = v.release();
    return NBP_OK;
    NBP_API_END(c)
}

nbp_status nbp_vms_destroy(nbp_vms *v) {
    if (!v) return NBP_ERR_INVALID;
    if (v->ctx) cudaSetDevice(v->ctx->dev);
    vms_free(v);
    return NBP_OK;
}

nbp_status nbp_vms_residual(nbp_vms *v, const double *vd, const double *vel, const double *p, const double *vtau,
                            const double *P, double *R) {
    VMS_BEGIN(v)
    begin_call(c);
    require(vd && vel && p && R && (P || c->lr.n_out == 0), NBP_ERR_INVALID, "nbp_vms_residual: null array");
    vms_residual_ctx(v, vd, vel, p, vtau, P, R);
    NBP_CUDA(cudaStreamSynchronize(c->s));
    return NBP_OK;
    VMS_END
}

nbp_status nbp_vms_tangent(nbp_vms *v, const double *vd, const double *vel, const double *p, const double *vtau,
                           double *a_val, double *b_val, double *c_val, double *d_val) {
    VMS_BEGIN(v)
    begin_call(c);
    require(vd && vel && p && a_val && b_val && c_val && d_val, NBP_ERR_INVALID, "nbp_vms_tangent: null array");
    vms_tangent(v->m, v->k, vd, vel, p, vtau, a_val, b_val, c_val, d_val, c->s);
    NBP_CUDA(cudaStreamSynchronize(c->s));
    return NBP_OK;
    VMS_END
}

nbp_status nbp_newton_step(nbp_vms *v, const nbp_rcr *rcr, const double *y_n, const double *yd_n, double *y,
                           double *yd, double *Pi_np1, const nbp_newton_opts *o, nbp_newton_info *info) {
    VMS_BEGIN(v)
    begin_call(c);
    using clk = std::chrono::steady_clock;
    const auto t_all = clk::now();
    require(y_n && yd_n && y && yd && o, NBP_ERR_INVALID, "nbp_newton_step: null argument");
    require(o->l_max >= 1 && o->nts >= 1 && o->tol_R >= 0 && o->tol_A >= 0 && o->pc_rebuild >= 0 &&
                o->pc_rebuild <= 4,
            NBP_ERR_INVALID, "nbp_newton_step: bad options");
    const int n_out = c->lr.n_out;
    nbp_rcr chk{};
    if (rcr) {
        chk = *rcr;
        chk.Q_n = chk.Rp;   // Q_n is computed here from y_n, not read
    }
    require(n_out == 0 || (rcr && rcr_params_ok(&chk)), NBP_ERR_INVALID, "nbp_newton_step: RCR parameters missing");
    vms_buffers(v);
    cudaStream_t s = c->s;
    const int N = c->N;
    const long long n = 4LL * N;
    const VmsConst &k = v->k;
    double *Qn = v->ob, *Q1 = v->ob + n_out, *Pn = v->ob + 2 * n_out, *P1 = v->ob + 3 * n_out;
    double *Pi1 = v->ob + 4 * n_out, *mk = v->ob + 5 * n_out, *rnew = v->ob + 6 * n_out, *Paf = v->ob + 7 * n_out;
    nbp_newton_info inf{};
    k_newton_predict<<<grid_for(n), 256, 0, s>>>(n, y_n, yd_n, (k.gm - 1.0) / k.gm, y, yd);
    NBP_LAUNCHED();
    nbp_rcr rl{};
    if (n_out) {
        rl = *rcr;
        rl.Q_n = Qn;
        launch_outlet_flows(n_out, c->lr.optr, c->lr.oidx, c->lr.oval, y_n, Qn, s);
        k_outlet_pn<<<(n_out + 127) / 128, 128, 0, s>>>(n_out, rcr->Rp, rcr->Pi_n, rcr->Pd, Qn, Pn);
        NBP_LAUNCHED();
    }
    double r0 = -1.0;
    for (int l = 1; l <= o->l_max; ++l) {
        auto t0 = clk::now();
        if (n_out) {                                                                      // steps 1-3
            NBP_CUDA(cudaMemsetAsync(v->bad, 0, sizeof(int), s));
            launch_outlet_flows(n_out, c->lr.optr, c->lr.oidx, c->lr.oval, y, Q1, s);
            launch_rcr_step(n_out, rl, Q1, k.dt, o->nts, P1, Pi1, mk, rnew, k.c, v->bad, s);
            k_outlet_paf<<<(n_out + 127) / 128, 128, 0, s>>>(n_out, Pn, P1, k.af, Paf);   // step 5
            NBP_LAUNCHED();
        }
        k_newton_stage<<<grid_for(n), 256, 0, s>>>(n, y_n, yd_n, y, yd, k.af, k.am, v->yaf, v->ydam);   // step 4
        NBP_LAUNCHED();
        vms_residual_ctx(v, v->ydam, v->yaf, v->yaf + 3LL * N, nullptr, n_out ? Paf : nullptr, v->R);   // step 6
        const double nr = norm2(v->R, n, v->part, s);
        inf.residual_s += std::chrono::duration<double>(clk::now() - t0).count();
        require(std::isfinite(nr), NBP_ERR_NAN, "nbp_newton_step: non-finite residual");
        if (r0 < 0) r0 = nr;
        inf.res0 = r0;
        inf.res = nr;
        if ((r0 > 0 && nr / r0 <= o->tol_R) || nr <= o->tol_A) { inf.converged = 1; break; }   // step 7
        t0 = clk::now();
        // preconditioner from this tangent (in full, or numerically on the
        // held aggregates), or the one held (lagged)
        const bool held = c->setup_done && c->HA.built && c->HS.built;
        const bool rebuild = o->pc_rebuild == 0 || (o->pc_rebuild == 1 && l == 1) || !held;
        const bool numeric = !rebuild && (o->pc_rebuild == 3 || (o->pc_rebuild == 4 && l == 1));
        vms_tangent(v->m, k, v->ydam, v->yaf, v->yaf + 3LL * N, nullptr, c->A.v, c->B.v, c->C.v, c->D.v, s);   // step 8
        if (rebuild || numeric) values_changed(c);
        else refresh_operators(c);
        if (n_out) {
            int bad = readback(v->bad, s);
            require(!bad, NBP_ERR_NAN, "nbp_newton_step: non-finite outlet stiffness m^k");
            std::vector<double> r(n_out);
            NBP_CUDA(cudaMemcpyAsync(c->lr.r, rnew, sizeof(double) * n_out, cudaMemcpyDeviceToDevice, s));
            NBP_CUDA(cudaMemcpyAsync(r.data(), rnew, sizeof(double) * n_out, cudaMemcpyDeviceToHost, s));
            NBP_CUDA(cudaStreamSynchronize(s));
            c->lr.r_host = r;
        }
        NBP_CUDA(cudaStreamSynchronize(s));
        inf.tangent_s += std::chrono::duration<double>(clk::now() - t0).count();
        t0 = clk::now();
        if (rebuild) {
            do_setup(c);
            inf.setups++;
        } else if (numeric) {
            do_setup(c, true);
            inf.numeric_setups++;
        }
        inf.setup_s += std::chrono::duration<double>(clk::now() - t0).count();
        t0 = clk::now();
        k_negate<<<grid_for(n), 256, 0, s>>>(n, v->R, v->rhs);
        NBP_LAUNCHED();
        nbp_info si{};
        const nbp_status st = solve_common(c, v->rhs, v->dx, nullptr, &si);   // step 9
        require(st == NBP_OK || st == NBP_NOT_CONVERGED, st, "nbp_newton_step: nested solve failed");
        inf.unconverged_solves += (st != NBP_OK);
        inf.outer_iters += si.outer_iters;
        inf.A_iters += si.A_iters;
        inf.S_iters += si.S_iters;
        inf.I_iters += si.I_iters;
        k_newton_update<<<grid_for(n), 256, 0, s>>>(N, v->m.dir, v->dx, k.gm * k.dt, y, yd);   // step 10
        NBP_LAUNCHED();
        inf.iters = l;
        inf.solve_s += std::chrono::duration<double>(clk::now() - t0).count();
    }
    if (Pi_np1 && n_out) NBP_CUDA(cudaMemcpyAsync(Pi_np1, Pi1, sizeof(double) * n_out, cudaMemcpyDeviceToDevice, s));
    NBP_CUDA(cudaStreamSynchronize(s));
    inf.total_s = std::chrono::duration<double>(clk::now() - t_all).count();
    if (info) *info = inf;
    return inf.converged ? NBP_OK : NBP_NOT_CONVERGED;
    VMS_END
}

}  // extern "C"
