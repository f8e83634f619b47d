/*
 * nbp_oracle.c -- plain, slow, FP64 CPU oracle of the nested block
 * preconditioned Krylov solve of the tangent [[A, B], [C, D]].
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark call this code; the product (the CUDA
 * library) never does, and it shares no code with it.
 *
 * What it computes, with the passage each part follows:
 *   - y = A x with A = A_sp + sum_k r_k a^k a^kT: the tangent block A = F + K
 *     with the resistance part K as a weighted sum of rank-one matrices
 *     (Sec. 2.5, definition of K); applied as a sparse product plus inner
 *     products (Sec. 3.3 remarks that the rank-one term acts by inner
 *     products).
 *   - Outer FGMRES(m), right preconditioned, variable preconditioner (Sec. 3,
 *     Saad 1993); stopping on ||r|| <= max(delta^r ||r_0||, delta^a) with
 *     x_0 = 0, restart every m steps, at most n_max iterations (Sec. 3.1,
 *     last paragraph before the SIMPLE section).
 *   - P_SCR^{-1} (Algorithm 3) and the matrix-free Schur product S x
 *     (Algorithm 2), with S = D - C A^{-1} B (Eq. of the block LDU
 *     factorisation, Sec. 3.1).
 *   - GMRES(m_A) with P_A on A and GMRES(m_S) with P_S = AMG(S_hat),
 *     S_hat = D - C diag(A)^{-1} B (Sec. 3.1).  Both are run in flexible form
 *     (the preconditioned directions are stored), which equals
 *     right-preconditioned GMRES in exact arithmetic for a fixed linear
 *     preconditioner.  P_S is applied on the right (the paper applies it on
 *     the left; right preconditioning keeps delta_S on the true residual).
 *   - P_A / P_S: an unsmoothed aggregation AMG V(1,1)-cycle with Chebyshev
 *     smoothing.  The paper uses BoomerAMG (Table 1) as prior art; the
 *     aggregation rule below is this project's, stated step by step:
 *       strength  sigma_ij = 0.5 (|A_ij|_F^2 + |A_ji|_F^2) / sqrt(|A_ii|_F^2 |A_jj|_F^2)
 *                 (squared Frobenius norms summed in row-major order, no
 *                 fused multiply-add), strong iff sigma_ij >= theta;
 *       matching  64 synchronous rounds: every unmatched node picks its
 *                 strongest unmatched strong neighbour (ties: smaller index),
 *                 mutual picks are matched; leftovers are singletons;
 *       passes    3 matching passes, pass k+1 on the aggregate graph of pass
 *                 k whose edge weight is the max of the member weights;
 *       numbering aggregates ordered by their smallest fine index;
 *       Galerkin  A_c = P^T A P with P = indicator (x) I_bs, each coarse
 *                 block the sequential sum of its fine blocks taken in
 *                 ascending (row, column) order;
 *       isolated  nodes with no strong connection (e.g. Dirichlet rows) are
 *                 left out of every aggregate (zero row of P);
 *       coarsest  dense LU with partial pivoting.
 *   - Chebyshev smoothing of degree k on D_b^{-1} A (D_b = block diagonal),
 *     interval [rho/10, rho] on AMG(A) and [rho/3, rho] on AMG(S_hat)
 *     (Saad, Iterative Methods, Alg. 12.1), rho the
 *     Gershgorin bound of D_b^{-1} A (largest absolute row sum); on the
 *     levels of AMG(A) the smaller of that bound and 1.1 x the spectral
 *     radius of the Hessenberg matrix of 20 Arnoldi steps on D_b^{-1} A from
 *     the vector of ones (the largest Ritz value magnitude, an estimate of
 *     the largest eigenvalue magnitude from below; the factor 1.1 keeps rho
 *     above it).  The Hessenberg spectral radius is lim ||H^m||^(1/m)
 *     (Gelfand), taken by repeated squaring.
 *   - RCR (three-element Windkessel) outlets, Sec. 2.1 / 2.4: one time step
 *     of dPi/dt = -Pi/(R_d C) + Q/C, P = R_p Q + Pi + P_d by the
 *     fourth-order Runge-Kutta scheme of Algorithm 1 (n_ts substeps, Q
 *     linear in time), and the stiffness m^k = dP_{n+1}/dQ_{n+1} by the
 *     central difference quotient of Sec. 2.5 (eps = max(eps_abs,
 *     eps_rel |Q|)).
 *
 * Vectors: x = [x_v (3N, node-interleaved); x_p (N)].
 * Build with -ffp-contract=off so that no multiply-add is fused, and with
 * -fopenmp: threads share only loops with independent iterations, and every
 * sum keeps one fixed order, so the results do not depend on the thread
 * count (OpenMP static scheduling with fixed-order reductions).
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXLEV 12
/* Loops whose iterations are independent (the rows of a sparse product,
 * elementwise vector updates, the prolongation, the restriction's per-
 * aggregate sums) run on all cores with OpenMP (static schedule) once they
 * exceed this length.  Every sum keeps one fixed order (inner products: see
 * dot()), so a result is the same bit for bit at any thread count. */
#define OR_PAR_MIN 32768
/* handshake rounds per matching pass; a round that adds no pair leaves the
 * state unchanged, so extra rounds after convergence are no-ops */
#define MATCH_ROUNDS 64

/* ----------------------------------------------------------------- types */
typedef struct {
    int nbr, nbc, br, bc; /* block rows / cols, block shape br x bc */
    int *rp, *ci;
    double *v;            /* br*bc values per block, row-major */
} bmat;

typedef struct {
    double rtol, rtol_A, rtol_S, rtol_I, atol;
    int m, m_A, m_S, nmax, nmax_A, nmax_S;
    int pc_A;           /* 0 AMG, 1 point Jacobi diag(A)^{-1} */
    int pc_S;           /* 0 AMG(S_hat), 1 none */
    int variant;        /* 0 P_SCR (Algorithm 3), 1 upper block-triangular [[A,B],[0,S]], 2 SIMPLE */
    int amg_max_levels, amg_coarse_max, cheb_degree;
    double theta;
    int amg_cycle;      /* 0 V-cycles; 1 K-cycle (two GCR steps on the coarse levels) on
                           AMG(S_hat); 2 K-cycle on both hierarchies */
    int amg_kdepth;     /* K-cycle on coarse levels 1..amg_kdepth, V-cycles below */
    int cheb_degree_S;  /* Chebyshev degree of the AMG(S_hat) smoother (cheb_degree: AMG(A)) */
    int cheb_degree_I;  /* Chebyshev degree of the AMG(A) cycle inside the inner A-solves of
                           Algorithm 2 (tolerance rtol_I); cheb_degree in every other A-solve */
} or_options;

typedef struct {
    int outer_iters;
    long long A_iters, S_iters, I_iters;
    long long n_A_solves, n_I_solves, n_S_solves;
    double rel_res_est, rel_res_true;
    int status;
} or_info;

typedef struct {
    int nlev, bs;
    bmat L[OR_MAXLEV];
    int *agg[OR_MAXLEV];    /* level l -> l+1 */
    int *mptr[OR_MAXLEV], *mem[OR_MAXLEV]; /* aggregate member lists */
    double *dinv[OR_MAXLEV];
    double rho[OR_MAXLEV];
    double *lu; int *piv; int nc; /* coarsest dense LU, nc = rows */
    double *bl[OR_MAXLEV], *xl[OR_MAXLEV], *rl[OR_MAXLEV], *dl[OR_MAXLEV];
    double *kr[OR_MAXLEV], *kz1[OR_MAXLEV], *kw1[OR_MAXLEV], *kz2[OR_MAXLEV], *kw2[OR_MAXLEV]; /* K-cycle */
    int cheb_degree, cycle, kdepth;
    double cheb_lo;         /* Chebyshev interval [rho / cheb_lo, rho] */
} amg;

typedef struct {
    int N;
    bmat A, B, C, D;        /* A: N x N blocks 3x3; B: N x N blocks 3x1; C: N x N blocks 1x3; D: N x N 1x1 */
    int n_out;
    int *out_ptr, *out_idx;
    double *out_val, *r;
    double *diagA;          /* scalar diagonal of A incl. rank-one terms (3N) */
    bmat Shat;
    amg amgA, amgS;
    int have_amgA, have_amgS;
    or_options opt;
    or_info info;
    double *wv1, *wv2, *wv3, *wp1, *wp2, *wp3, *wp4;
} or_ctx;

/* --------------------------------------------------------------- helpers */
static void *xmalloc(size_t n) {
    void *p = malloc(n ? n : 1);
    if (!p) { fprintf(stderr, "oracle: out of memory\n"); abort(); }
    return p;
}
static double *dvec(size_t n) { return (double *)calloc(n ? n : 1, sizeof(double)); }

/* Inner product in a fixed order: a sequential sum over each run of
 * OR_DOT_BLOCK consecutive entries, then the run sums added in ascending
 * order.  The runs may be summed by different threads; the order, and so the
 * result, is the same at any thread count (a vector of at most OR_DOT_BLOCK
 * entries is one plain sequential sum). */
#define OR_DOT_BLOCK 4096
static double dot(int n, const double *a, const double *b) {
    const int nb = (n + OR_DOT_BLOCK - 1) / OR_DOT_BLOCK;
    if (nb <= 1) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += a[i] * b[i];
        return s;
    }
    double *part = (double *)malloc(sizeof(double) * (size_t)nb);
    if (!part) { fprintf(stderr, "oracle: out of memory\n"); abort(); }
#pragma omp parallel for schedule(static) if ((n) > OR_PAR_MIN)
    for (int k = 0; k < nb; ++k) {
        const int lo = k * OR_DOT_BLOCK, hi = lo + OR_DOT_BLOCK < n ? lo + OR_DOT_BLOCK : n;
        double s = 0.0;
        for (int i = lo; i < hi; ++i) s += a[i] * b[i];
        part[k] = s;
    }
    double s = 0.0;
    for (int k = 0; k < nb; ++k) s += part[k];
    free(part);
    return s;
}
static double nrm2(int n, const double *a) { return sqrt(dot(n, a, a)); }

static void bmat_copy(bmat *dst, int nbr, int nbc, int br, int bc, const int *rp, const int *ci, const double *v) {
    dst->nbr = nbr; dst->nbc = nbc; dst->br = br; dst->bc = bc;
    int nnz = rp[nbr];
    dst->rp = (int *)xmalloc(sizeof(int) * (nbr + 1));
    dst->ci = (int *)xmalloc(sizeof(int) * (size_t)nnz);
    dst->v = (double *)xmalloc(sizeof(double) * (size_t)nnz * br * bc);
    memcpy(dst->rp, rp, sizeof(int) * (nbr + 1));
    memcpy(dst->ci, ci, sizeof(int) * (size_t)nnz);
    memcpy(dst->v, v, sizeof(double) * (size_t)nnz * br * bc);
}
static void bmat_free(bmat *m) { free(m->rp); free(m->ci); free(m->v); memset(m, 0, sizeof(*m)); }

/* y = M x (block sparse product, plain row loop) */
static void spmv(const bmat *M, const double *x, double *y) {
    int br = M->br, bc = M->bc, bs = br * bc;
#pragma omp parallel for schedule(static) if ((M->nbr) > OR_PAR_MIN)
    for (int i = 0; i < M->nbr; ++i) {
        double acc[3] = {0.0, 0.0, 0.0};
        for (int e = M->rp[i]; e < M->rp[i + 1]; ++e) {
            const double *blk = M->v + (size_t)e * bs;
            const double *xj = x + (size_t)M->ci[e] * bc;
            for (int r = 0; r < br; ++r)
                for (int c = 0; c < bc; ++c) acc[r] += blk[r * bc + c] * xj[c];
        }
        for (int r = 0; r < br; ++r) y[(size_t)i * br + r] = acc[r];
    }
}

/* ---------------------------------------------------- operator blocks */
/* y = A x = A_sp x + sum_k r_k a^k (a^kT x)   (Sec. 2.5, A = F + K) */
void or_apply_A(or_ctx *c, const double *x, double *y) {
    spmv(&c->A, x, y);
    for (int k = 0; k < c->n_out; ++k) {
        double s = 0.0;
        for (int e = c->out_ptr[k]; e < c->out_ptr[k + 1]; ++e) s += c->out_val[e] * x[c->out_idx[e]];
        double f = c->r[k] * s;
        for (int e = c->out_ptr[k]; e < c->out_ptr[k + 1]; ++e) y[c->out_idx[e]] += f * c->out_val[e];
    }
}
void or_apply_B(or_ctx *c, const double *xp, double *yv) { spmv(&c->B, xp, yv); }
void or_apply_C(or_ctx *c, const double *xv, double *yp) { spmv(&c->C, xv, yp); }
void or_apply_D(or_ctx *c, const double *xp, double *yp) { spmv(&c->D, xp, yp); }

/* y = [[A, B], [C, D]] x   (tangent of Sec. 2.5 / block system of Sec. 3) */
void or_apply_full(or_ctx *c, const double *x, double *y) {
    int nv = 3 * c->N, np = c->N;
    const double *xv = x, *xp = x + nv;
    double *yv = y, *yp = y + nv;
    or_apply_A(c, xv, yv);
    spmv(&c->B, xp, c->wv1);
#pragma omp parallel for schedule(static) if ((nv) > OR_PAR_MIN)
    for (int i = 0; i < nv; ++i) yv[i] += c->wv1[i];
    spmv(&c->C, xv, yp);
    spmv(&c->D, xp, c->wp1);
#pragma omp parallel for schedule(static) if ((np) > OR_PAR_MIN)
    for (int i = 0; i < np; ++i) yp[i] += c->wp1[i];
}

/* ------------------------------------------------------ GMRES / FGMRES */
typedef void (*linop)(void *ctx, const double *x, double *y);

/* Restarted flexible GMRES with right preconditioning (Saad 1993):
 * modified Gram-Schmidt Arnoldi, Givens rotations on the Hessenberg matrix,
 * x_0 = 0, stop when the residual estimate |g_{j+1}| <= max(rtol ||b||, atol)
 * or after nmax iterations.  If check_true, convergence is confirmed on the
 * true residual b - op(x), and a failed check restarts.  Returns 0 when
 * converged, 1 otherwise; *its = iterations, *rel = final relative residual
 * (estimate, or true if check_true). */
static int fgmres(int n, linop op, void *opc, linop pc, void *pcc, const double *b, double *x,
                  double rtol, double atol, int m, int nmax, int check_true, int *its_out, double *rel_out,
                  double *rel_true_out) {
    double *V = dvec((size_t)n * (m + 1));
    double *Z = dvec((size_t)n * m);
    double *H = dvec((size_t)(m + 1) * m);
    double *cs = dvec(m), *sn = dvec(m), *g = dvec(m + 1), *y = dvec(m);
    double *r = dvec(n), *w = dvec(n);
#pragma omp parallel for schedule(static) if ((n) > OR_PAR_MIN)
    for (int i = 0; i < n; ++i) { x[i] = 0.0; r[i] = b[i]; }
    double bnorm = nrm2(n, b);
    double tol = fmax(rtol * bnorm, atol);
    double beta = bnorm, res = bnorm;
    int its = 0, conv = (beta <= tol);
    double rel_true = (bnorm > 0) ? 1.0 : 0.0;
    while (!conv && its < nmax) {
        #pragma omp parallel for schedule(static) if ((n) > OR_PAR_MIN)
        for (int i = 0; i < n; ++i) V[i] = r[i] / beta;
        memset(g, 0, sizeof(double) * (m + 1));
        g[0] = beta;
        int jend = 0;
        for (int j = 0; j < m && its < nmax; ++j) {
            double *vj = V + (size_t)j * n, *zj = Z + (size_t)j * n;
            if (pc) pc(pcc, vj, zj); else memcpy(zj, vj, sizeof(double) * n);
            op(opc, zj, w);
            for (int i = 0; i <= j; ++i) {           /* modified Gram-Schmidt */
                double h = dot(n, w, V + (size_t)i * n);
                H[i * m + j] = h;
                #pragma omp parallel for schedule(static) if ((n) > OR_PAR_MIN)
                for (int t = 0; t < n; ++t) w[t] -= h * V[(size_t)i * n + t];
            }
            double hn = nrm2(n, w);
            H[(j + 1) * m + j] = hn;
            for (int i = 0; i < j; ++i) {             /* previous rotations */
                double a = H[i * m + j], bb = H[(i + 1) * m + j];
                H[i * m + j] = cs[i] * a + sn[i] * bb;
                H[(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
            }
            double a = H[j * m + j], bb = H[(j + 1) * m + j];
            double den = hypot(a, bb);
            if (den == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
            else { cs[j] = a / den; sn[j] = bb / den; }
            H[j * m + j] = den;
            H[(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            res = fabs(g[j + 1]);
            ++its;
            jend = j + 1;
            if (hn != 0.0) {
                #pragma omp parallel for schedule(static) if ((n) > OR_PAR_MIN)
                for (int t = 0; t < n; ++t) V[(size_t)(j + 1) * n + t] = w[t] / hn;
            }
            if (res <= tol || hn == 0.0) break;
        }
        /* back substitution H y = g */
        for (int i = jend - 1; i >= 0; --i) {
            double s = g[i];
            for (int k = i + 1; k < jend; ++k) s -= H[i * m + k] * y[k];
            y[i] = (H[i * m + i] != 0.0) ? s / H[i * m + i] : 0.0;
        }
        for (int i = 0; i < jend; ++i) {
            #pragma omp parallel for schedule(static) if ((n) > OR_PAR_MIN)
            for (int t = 0; t < n; ++t) x[t] += y[i] * Z[(size_t)i * n + t];
        }
        int est_conv = (res <= tol);
        if (est_conv && !check_true) { conv = 1; break; }
        /* true residual: restart vector, or the confirmation of convergence */
        op(opc, x, w);
        #pragma omp parallel for schedule(static) if ((n) > OR_PAR_MIN)
        for (int t = 0; t < n; ++t) r[t] = b[t] - w[t];
        beta = nrm2(n, r);
        res = beta;
        rel_true = bnorm > 0 ? beta / bnorm : 0.0;
        if (beta <= tol) { conv = 1; break; }
        if (beta == 0.0) break;
    }
    *its_out = its;
    *rel_out = bnorm > 0 ? res / bnorm : 0.0;
    if (rel_true_out) *rel_true_out = rel_true;
    free(V); free(Z); free(H); free(cs); free(sn); free(g); free(y); free(r); free(w);
    return conv ? 0 : 1;
}

/* ------------------------------------------------------ aggregation AMG */
/* squared Frobenius norm, row-major sequential sum */
static double fnorm2(const double *blk, int nb) {
    double s = blk[0] * blk[0];
    for (int t = 1; t < nb; ++t) s = s + blk[t] * blk[t];
    return s;
}

static int find_entry(const bmat *M, int i, int j) {
    int lo = M->rp[i], hi = M->rp[i + 1] - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        if (M->ci[mid] == j) return mid;
        if (M->ci[mid] < j) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

typedef struct { int n; int *p; int *j; double *w; } wgraph;
static void wgraph_free(wgraph *g) { free(g->p); free(g->j); free(g->w); }

/* One matching pass: MATCH_ROUNDS synchronous handshake rounds; returns number of
 * aggregates and writes map[u] (aggregates numbered by smallest member). */
static int match_pass(const wgraph *G, double theta, int *map) {
    int n = G->n;
    int *mate = (int *)xmalloc(sizeof(int) * n), *pick = (int *)xmalloc(sizeof(int) * n);
    for (int u = 0; u < n; ++u) mate[u] = -1;
    for (int round = 0; round < MATCH_ROUNDS; ++round) {
        for (int u = 0; u < n; ++u) {
            pick[u] = -1;
            if (mate[u] >= 0) continue;
            double best = 0.0;
            for (int e = G->p[u]; e < G->p[u + 1]; ++e) {
                int v = G->j[e];
                if (v == u || mate[v] >= 0) continue;
                double w = G->w[e];
                if (!(w >= theta)) continue;
                if (pick[u] < 0 || w > best || (w == best && v < pick[u])) { best = w; pick[u] = v; }
            }
        }
        for (int u = 0; u < n; ++u) {
            int v = pick[u];
            if (v >= 0 && pick[v] == u) mate[u] = v;
        }
    }
    int nc = 0;
    for (int u = 0; u < n; ++u) {
        int root = (mate[u] >= 0 && mate[u] < u) ? mate[u] : u;
        if (root == u) map[u] = nc++;
    }
    for (int u = 0; u < n; ++u)
        if (mate[u] >= 0 && mate[u] < u) map[u] = map[mate[u]];
    free(mate); free(pick);
    return nc;
}

static int cmp_int(const void *a, const void *b) { int x = *(const int *)a, y = *(const int *)b; return (x > y) - (x < y); }

/* Aggregate graph: edge weight = max of member edge weights (I != J). */
static void coarse_graph(const wgraph *G, const int *map, int nc, wgraph *Gc) {
    int n = G->n;
    int *cnt = (int *)calloc((size_t)nc + 1, sizeof(int));
    for (int u = 0; u < n; ++u) cnt[map[u] + 1]++;
    for (int I = 0; I < nc; ++I) cnt[I + 1] += cnt[I];
    int *mem = (int *)xmalloc(sizeof(int) * n), *fill = (int *)xmalloc(sizeof(int) * nc);
    memcpy(fill, cnt, sizeof(int) * nc);
    for (int u = 0; u < n; ++u) mem[fill[map[u]]++] = u;
    int *marker = (int *)xmalloc(sizeof(int) * nc);
    for (int I = 0; I < nc; ++I) marker[I] = -1;
    size_t cap = (size_t)G->p[n] + 1;
    Gc->n = nc;
    Gc->p = (int *)xmalloc(sizeof(int) * (nc + 1));
    Gc->j = (int *)xmalloc(sizeof(int) * cap);
    Gc->w = (double *)xmalloc(sizeof(double) * cap);
    int pos = 0;
    for (int I = 0; I < nc; ++I) {
        Gc->p[I] = pos;
        int start = pos;
        for (int t = cnt[I]; t < cnt[I + 1]; ++t) {
            int u = mem[t];
            for (int e = G->p[u]; e < G->p[u + 1]; ++e) {
                int J = map[G->j[e]];
                if (J == I) continue;
                if (marker[J] < start) { marker[J] = pos; Gc->j[pos] = J; Gc->w[pos] = G->w[e]; ++pos; }
                else if (G->w[e] > Gc->w[marker[J]]) Gc->w[marker[J]] = G->w[e];
            }
        }
        /* sort row by J (insertion sort keeps weights attached) */
        for (int a = start + 1; a < pos; ++a) {
            int jj = Gc->j[a]; double ww = Gc->w[a]; int b = a - 1;
            while (b >= start && Gc->j[b] > jj) { Gc->j[b + 1] = Gc->j[b]; Gc->w[b + 1] = Gc->w[b]; --b; }
            Gc->j[b + 1] = jj; Gc->w[b + 1] = ww;
        }
    }
    Gc->p[nc] = pos;
    free(cnt); free(mem); free(fill); free(marker);
}

/* Strength graph of a level matrix (off-diagonal pattern, symmetric weights). */
static void strength_graph(const bmat *M, wgraph *G) {
    int n = M->nbr, nb = M->br * M->bc;
    double *dn = dvec(n);
    for (int i = 0; i < n; ++i) {
        int e = find_entry(M, i, i);
        dn[i] = (e >= 0) ? fnorm2(M->v + (size_t)e * nb, nb) : 0.0;
    }
    G->n = n;
    G->p = (int *)xmalloc(sizeof(int) * (n + 1));
    G->j = (int *)xmalloc(sizeof(int) * (size_t)M->rp[n] + 1);
    G->w = (double *)xmalloc(sizeof(double) * (size_t)M->rp[n] + 1);
    int pos = 0;
    for (int i = 0; i < n; ++i) {
        G->p[i] = pos;
        for (int e = M->rp[i]; e < M->rp[i + 1]; ++e) {
            int j = M->ci[e];
            if (j == i) continue;
            double fij = fnorm2(M->v + (size_t)e * nb, nb);
            int et = find_entry(M, j, i);
            double fji = (et >= 0) ? fnorm2(M->v + (size_t)et * nb, nb) : 0.0;
            double d = dn[i] * dn[j];
            double w = (fij + fji) * 0.5;
            G->j[pos] = j;
            G->w[pos] = (d > 0.0) ? w / sqrt(d) : 0.0;
            ++pos;
        }
    }
    G->p[n] = pos;
    free(dn);
}

/* Three matching passes -> fine-to-aggregate map; returns aggregate count. */
static int aggregate(const bmat *M, double theta, int *agg) {
    wgraph G;
    strength_graph(M, &G);
    int n = M->nbr;
    /* isolated nodes: no strong off-diagonal connection at all */
    int *iso = (int *)xmalloc(sizeof(int) * (n ? n : 1));
    for (int i = 0; i < n; ++i) {
        iso[i] = 1;
        for (int e = G.p[i]; e < G.p[i + 1]; ++e)
            if (G.w[e] >= theta) { iso[i] = 0; break; }
    }
    for (int i = 0; i < n; ++i) agg[i] = i;
    int nc = n;
    int *map = (int *)xmalloc(sizeof(int) * n);
    for (int pass = 0; pass < 3; ++pass) {
        int nn = match_pass(&G, theta, map);
        for (int i = 0; i < n; ++i) agg[i] = map[agg[i]];
        wgraph Gc;
        coarse_graph(&G, map, nn, &Gc);
        wgraph_free(&G);
        G = Gc;
        nc = nn;
    }
    wgraph_free(&G);
    free(map);
    /* isolated nodes stay singletons through every pass; drop them (zero row
     * of P) and renumber the remaining aggregates in the same order */
    int *keep = (int *)calloc((size_t)nc + 1, sizeof(int));
    for (int i = 0; i < n; ++i)
        if (!iso[i]) keep[agg[i]] = 1;
    int *newid = (int *)xmalloc(sizeof(int) * ((size_t)nc + 1));
    int m = 0;
    for (int I = 0; I < nc; ++I) newid[I] = keep[I] ? m++ : -1;
    for (int i = 0; i < n; ++i) agg[i] = iso[i] ? -1 : newid[agg[i]];
    free(keep); free(newid); free(iso);
    return m;
}

/* Galerkin A_c = P^T A P, P = aggregate indicator (x) I_bs. */
static void galerkin(const bmat *M, const int *agg, int nc, bmat *Mc) {
    int n = M->nbr, nb = M->br * M->bc;
    int *cnt = (int *)calloc((size_t)nc + 1, sizeof(int));
    for (int i = 0; i < n; ++i)
        if (agg[i] >= 0) cnt[agg[i] + 1]++;
    for (int I = 0; I < nc; ++I) cnt[I + 1] += cnt[I];
    int *mem = (int *)xmalloc(sizeof(int) * (n ? n : 1)), *fill = (int *)xmalloc(sizeof(int) * (nc ? nc : 1));
    memcpy(fill, cnt, sizeof(int) * nc);
    for (int i = 0; i < n; ++i)                           /* ascending i within each aggregate */
        if (agg[i] >= 0) mem[fill[agg[i]]++] = i;
    int *marker = (int *)xmalloc(sizeof(int) * nc);
    for (int I = 0; I < nc; ++I) marker[I] = -1;
    size_t cap = (size_t)M->rp[n] + 1;
    int *ci = (int *)xmalloc(sizeof(int) * cap);
    double *v = (double *)xmalloc(sizeof(double) * cap * nb);
    Mc->nbr = nc; Mc->nbc = nc; Mc->br = M->br; Mc->bc = M->bc;
    Mc->rp = (int *)xmalloc(sizeof(int) * (nc + 1));
    int pos = 0;
    for (int I = 0; I < nc; ++I) {
        Mc->rp[I] = pos;
        int start = pos;
        for (int t = cnt[I]; t < cnt[I + 1]; ++t) {
            int i = mem[t];
            for (int e = M->rp[i]; e < M->rp[i + 1]; ++e) {
                int J = agg[M->ci[e]];
                if (J < 0) continue;
                const double *blk = M->v + (size_t)e * nb;
                if (marker[J] < start) {
                    marker[J] = pos; ci[pos] = J;
                    for (int q = 0; q < nb; ++q) v[(size_t)pos * nb + q] = blk[q];
                    ++pos;
                } else {
                    double *dst = v + (size_t)marker[J] * nb;
                    for (int q = 0; q < nb; ++q) dst[q] = dst[q] + blk[q];
                }
            }
        }
        /* sort the row by column, moving blocks */
        for (int a = start + 1; a < pos; ++a) {
            int jj = ci[a];
            double tmp[9];
            memcpy(tmp, v + (size_t)a * nb, sizeof(double) * nb);
            int b = a - 1;
            while (b >= start && ci[b] > jj) {
                ci[b + 1] = ci[b];
                memcpy(v + (size_t)(b + 1) * nb, v + (size_t)b * nb, sizeof(double) * nb);
                --b;
            }
            ci[b + 1] = jj;
            memcpy(v + (size_t)(b + 1) * nb, tmp, sizeof(double) * nb);
        }
    }
    Mc->rp[nc] = pos;
    Mc->ci = ci; Mc->v = v;
    free(cnt); free(mem); free(fill); free(marker);
}

/* inverse of the bs x bs diagonal blocks (adjugate for 3x3) */
static void block_diag_inv(const bmat *M, double *dinv) {
    int n = M->nbr, bs = M->br, nb = bs * bs;
    for (int i = 0; i < n; ++i) {
        int e = find_entry(M, i, i);
        double *o = dinv + (size_t)i * nb;
        if (bs == 1) { double a = (e >= 0) ? M->v[e] : 0.0; o[0] = (a != 0.0) ? 1.0 / a : 0.0; continue; }
        double z[9] = {0};
        const double *a = (e >= 0) ? M->v + (size_t)e * 9 : z;
        double c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8], c02 = a[3] * a[7] - a[4] * a[6];
        double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
        if (det == 0.0) { memset(o, 0, sizeof(double) * 9); continue; }
        double id = 1.0 / det;
        o[0] = c00 * id; o[1] = (a[2] * a[7] - a[1] * a[8]) * id; o[2] = (a[1] * a[5] - a[2] * a[4]) * id;
        o[3] = c01 * id; o[4] = (a[0] * a[8] - a[2] * a[6]) * id; o[5] = (a[2] * a[3] - a[0] * a[5]) * id;
        o[6] = c02 * id; o[7] = (a[1] * a[6] - a[0] * a[7]) * id; o[8] = (a[0] * a[4] - a[1] * a[3]) * id;
    }
}

static void apply_dinv(int n, int bs, const double *dinv, const double *r, double *z) {
    int nb = bs * bs;
#pragma omp parallel for schedule(static) if ((n) > OR_PAR_MIN)
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < bs; ++a) {
            double s = 0.0;
            for (int b = 0; b < bs; ++b) s += dinv[(size_t)i * nb + a * bs + b] * r[(size_t)i * bs + b];
            z[(size_t)i * bs + a] = s;
        }
}

/* Dense LU with partial pivoting (Golub & Van Loan, Alg. 3.4.1) */
static void dense_lu(int n, double *a, int *piv) {
    for (int k = 0; k < n; ++k) {
        int p = k; double mx = fabs(a[(size_t)k * n + k]);
        for (int i = k + 1; i < n; ++i) if (fabs(a[(size_t)i * n + k]) > mx) { mx = fabs(a[(size_t)i * n + k]); p = i; }
        piv[k] = p;
        if (p != k) for (int j = 0; j < n; ++j) { double t = a[(size_t)k * n + j]; a[(size_t)k * n + j] = a[(size_t)p * n + j]; a[(size_t)p * n + j] = t; }
        double d = a[(size_t)k * n + k];
        if (d == 0.0) continue;
        for (int i = k + 1; i < n; ++i) {
            double l = a[(size_t)i * n + k] / d;
            a[(size_t)i * n + k] = l;
            for (int j = k + 1; j < n; ++j) a[(size_t)i * n + j] -= l * a[(size_t)k * n + j];
        }
    }
}
static void dense_lu_solve(int n, const double *a, const int *piv, const double *b, double *x) {
    for (int i = 0; i < n; ++i) x[i] = b[i];
    for (int k = 0; k < n; ++k) { int p = piv[k]; if (p != k) { double t = x[k]; x[k] = x[p]; x[p] = t; } }
    for (int i = 0; i < n; ++i) for (int j = 0; j < i; ++j) x[i] -= a[(size_t)i * n + j] * x[j];
    for (int i = n - 1; i >= 0; --i) {
        for (int j = i + 1; j < n; ++j) x[i] -= a[(size_t)i * n + j] * x[j];
        x[i] = (a[(size_t)i * n + i] != 0.0) ? x[i] / a[(size_t)i * n + i] : 0.0;
    }
}

/* Upper bound of the spectral radius of D_b^{-1} A (Gershgorin): the largest
 * absolute row sum of D_b^{-1} A, each row summed in ascending column order. */
static double gershgorin_rho(const bmat *M, const double *dinv) {
    int bs = M->br, nb = bs * bs;
    double rho = 0.0;
    for (int i = 0; i < M->nbr; ++i) {
        const double *di = dinv + (size_t)i * nb;
        for (int a = 0; a < bs; ++a) {
            double s = 0.0;
            for (int e = M->rp[i]; e < M->rp[i + 1]; ++e) {
                const double *blk = M->v + (size_t)e * nb;
                for (int c = 0; c < bs; ++c) {
                    double t = 0.0;
                    for (int k = 0; k < bs; ++k) t += di[a * bs + k] * blk[k * bs + c];
                    s += fabs(t);
                }
            }
            if (s > rho) rho = s;
        }
    }
    return rho;
}

/* Spectral radius of the k x k matrix H (row-major) by Gelfand's formula
 * rho = lim ||H^m||_F^(1/m), with m = 2^40 reached by squaring; each square
 * is renormalised and the scale carried as a logarithm. */
static double spectral_radius_gelfand(int k, const double *H) {
    double *M = dvec((size_t)k * k), *T = dvec((size_t)k * k);
    double s = 0.0;
    for (int i = 0; i < k * k; ++i) s += H[i] * H[i];
    s = sqrt(s);
    if (s == 0.0) { free(M); free(T); return 0.0; }
    for (int i = 0; i < k * k; ++i) M[i] = H[i] / s;
    double logscale = log(s);   /* H^(2^q) = exp(logscale) M */
    const int Q = 40;
    for (int q = 0; q < Q; ++q) {
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) {
                double t = 0.0;
                for (int l = 0; l < k; ++l) t += M[i * k + l] * M[l * k + j];
                T[i * k + j] = t;
            }
        double n2 = 0.0;
        for (int i = 0; i < k * k; ++i) n2 += T[i] * T[i];
        const double n = sqrt(n2);
        if (n == 0.0) { free(M); free(T); return 0.0; }   /* nilpotent */
        for (int i = 0; i < k * k; ++i) M[i] = T[i] / n;
        logscale = 2.0 * logscale + log(n);
    }
    free(M); free(T);
    return exp(logscale / ldexp(1.0, Q));
}

/* 20 Arnoldi steps (classical Gram-Schmidt, two passes) on D_b^{-1} A from
 * the normalised vector of ones; returns the spectral radius of the square
 * Hessenberg matrix (stops early on an invariant subspace). */
#define RHO_ARNOLDI_STEPS 20
static double arnoldi_rho(const bmat *M, const double *dinv) {
    const int bs = M->br, nb = bs * bs, n = M->nbr * bs, K = RHO_ARNOLDI_STEPS;
    double *V = dvec((size_t)n * (K + 1)), *w = dvec(n), *t = dvec(n);
    double Hk[RHO_ARNOLDI_STEPS * RHO_ARNOLDI_STEPS];
    memset(Hk, 0, sizeof(Hk));
    for (int i = 0; i < n; ++i) V[i] = 1.0 / sqrt((double)n);
    int k = K;
    for (int j = 0; j < K; ++j) {
        spmv(M, V + (size_t)j * n, t);
        for (int r = 0; r < M->nbr; ++r)          /* w = D_b^{-1} (A v_j) */
            for (int a = 0; a < bs; ++a) {
                double u = 0.0;
                for (int c = 0; c < bs; ++c) u += dinv[(size_t)r * nb + a * bs + c] * t[(size_t)r * bs + c];
                w[(size_t)r * bs + a] = u;
            }
        for (int pass = 0; pass < 2; ++pass) {
            double h[RHO_ARNOLDI_STEPS + 1];
            for (int i = 0; i <= j; ++i) {
                double u = 0.0;
                for (int e = 0; e < n; ++e) u += V[(size_t)i * n + e] * w[e];
                h[i] = u;
            }
            for (int i = 0; i <= j; ++i) {
                for (int e = 0; e < n; ++e) w[e] -= h[i] * V[(size_t)i * n + e];
                Hk[i * K + j] += h[i];
            }
        }
        double nrm = 0.0;
        for (int e = 0; e < n; ++e) nrm += w[e] * w[e];
        nrm = sqrt(nrm);
        if (j + 1 < K) Hk[(j + 1) * K + j] = nrm;
        if (nrm == 0.0) { k = j + 1; break; }
        for (int e = 0; e < n; ++e) V[(size_t)(j + 1) * n + e] = w[e] / nrm;
    }
    double Hs[RHO_ARNOLDI_STEPS * RHO_ARNOLDI_STEPS];
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) Hs[i * k + j] = Hk[i * K + j];
    const double r = spectral_radius_gelfand(k, Hs);
    free(V); free(w); free(t);
    return r;
}

/* tight_rho: Chebyshev bound from the Arnoldi estimate (AMG(A)); else the
 * Gershgorin bound (AMG(S_hat)).  keep: the aggregate maps of an earlier
 * hierarchy of the same pattern to build on instead of aggregating again
 * (the numeric re-setup; everything else is computed from the new values);
 * its maps are moved into H. */
static void amg_build(amg *H, const bmat *fine, const or_options *o, int kcycle, int degree, int tight_rho,
                      double lodiv, amg *keep) {
    memset(H, 0, sizeof(*H));
    H->cheb_lo = lodiv;
    H->bs = fine->br;
    H->cheb_degree = degree;
    H->cycle = kcycle;
    H->kdepth = o->amg_kdepth;
    bmat_copy(&H->L[0], fine->nbr, fine->nbc, fine->br, fine->bc, fine->rp, fine->ci, fine->v);
    int l = 0;
    while (keep ? (l + 1 < keep->nlev) : (H->L[l].nbr > o->amg_coarse_max && l + 1 < o->amg_max_levels && l + 1 < OR_MAXLEV)) {
        int n = H->L[l].nbr, nc;
        if (keep) {   /* the kept map and its coarse size */
            H->agg[l] = keep->agg[l];
            keep->agg[l] = NULL;
            nc = keep->L[l + 1].nbr;
        } else {
            H->agg[l] = (int *)xmalloc(sizeof(int) * n);
            nc = aggregate(&H->L[l], o->theta, H->agg[l]);
            if (nc >= n || nc == 0) { free(H->agg[l]); H->agg[l] = NULL; break; }
        }
        galerkin(&H->L[l], H->agg[l], nc, &H->L[l + 1]);
        H->mptr[l] = (int *)calloc((size_t)nc + 1, sizeof(int));   /* members of each aggregate, ascending */
        H->mem[l] = (int *)xmalloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
        for (int i = 0; i < n; ++i) if (H->agg[l][i] >= 0) H->mptr[l][H->agg[l][i] + 1]++;
        for (int I = 0; I < nc; ++I) H->mptr[l][I + 1] += H->mptr[l][I];
        {
            int *fillp = (int *)xmalloc(sizeof(int) * (size_t)(nc > 0 ? nc : 1));
            memcpy(fillp, H->mptr[l], sizeof(int) * (size_t)nc);
            for (int i = 0; i < n; ++i) if (H->agg[l][i] >= 0) H->mem[l][fillp[H->agg[l][i]]++] = i;
            free(fillp);
        }
        ++l;
    }
    H->nlev = l + 1;
    for (int k = 0; k < H->nlev; ++k) {
        int n = H->L[k].nbr, bs = H->bs;
        H->bl[k] = dvec((size_t)n * bs); H->xl[k] = dvec((size_t)n * bs);
        H->rl[k] = dvec((size_t)n * bs); H->dl[k] = dvec((size_t)n * bs);
        H->kr[k] = dvec((size_t)n * bs); H->kz1[k] = dvec((size_t)n * bs); H->kw1[k] = dvec((size_t)n * bs);
        H->kz2[k] = dvec((size_t)n * bs); H->kw2[k] = dvec((size_t)n * bs);
        if (k + 1 < H->nlev) {
            H->dinv[k] = dvec((size_t)n * bs * bs);
            block_diag_inv(&H->L[k], H->dinv[k]);
            const double g = gershgorin_rho(&H->L[k], H->dinv[k]);
            const double a = tight_rho ? 1.1 * arnoldi_rho(&H->L[k], H->dinv[k]) : g;
            H->rho[k] = a < g ? a : g;
        }
    }
    /* coarsest: dense LU */
    bmat *Lc = &H->L[H->nlev - 1];
    int nc = Lc->nbr * H->bs, bs = H->bs;
    H->nc = nc;
    H->lu = dvec((size_t)nc * nc);
    H->piv = (int *)xmalloc(sizeof(int) * (nc ? nc : 1));
    for (int i = 0; i < Lc->nbr; ++i)
        for (int e = Lc->rp[i]; e < Lc->rp[i + 1]; ++e)
            for (int a = 0; a < bs; ++a)
                for (int b = 0; b < bs; ++b)
                    H->lu[(size_t)(i * bs + a) * nc + (size_t)Lc->ci[e] * bs + b] += Lc->v[(size_t)e * bs * bs + a * bs + b];
    dense_lu(nc, H->lu, H->piv);
}

static void amg_free(amg *H) {
    for (int k = 0; k < H->nlev; ++k) {
        bmat_free(&H->L[k]);
        free(H->agg[k]); free(H->mptr[k]); free(H->mem[k]); free(H->dinv[k]); free(H->bl[k]); free(H->xl[k]); free(H->rl[k]); free(H->dl[k]);
        free(H->kr[k]); free(H->kz1[k]); free(H->kw1[k]); free(H->kz2[k]); free(H->kw2[k]);
    }
    free(H->lu); free(H->piv);
    memset(H, 0, sizeof(*H));
}

/* Chebyshev smoothing, degree k, on D^{-1} A x = D^{-1} b, interval
 * [rho/10, 1.1 rho]; x updated in place (Saad, Alg. 12.1). */
static void chebyshev(const bmat *M, const double *dinv, double rho, double lodiv, int k, const double *b, double *x,
                      double *r, double *d, int x_is_zero) {
    int n = M->nbr * M->br;
    double lmax = rho, lmin = rho / lodiv;
    double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
    double sigma = theta / delta, rho_old = 1.0 / sigma;
    double *t = dvec(n);
    if (x_is_zero) memcpy(r, b, sizeof(double) * n);
    else {
        spmv(M, x, t);
#pragma omp parallel for schedule(static) if ((n) > OR_PAR_MIN)
        for (int i = 0; i < n; ++i) r[i] = b[i] - t[i];
    }
    apply_dinv(M->nbr, M->br, dinv, r, t);
#pragma omp parallel for schedule(static) if ((n) > OR_PAR_MIN)
    for (int i = 0; i < n; ++i) d[i] = t[i] / theta;
    for (int it = 0; it < k; ++it) {
        #pragma omp parallel for schedule(static) if ((n) > OR_PAR_MIN)
        for (int i = 0; i < n; ++i) x[i] += d[i];
        if (it + 1 == k) break;
        spmv(M, x, t);
        #pragma omp parallel for schedule(static) if ((n) > OR_PAR_MIN)
        for (int i = 0; i < n; ++i) r[i] = b[i] - t[i];
        double rho_new = 1.0 / (2.0 * sigma - rho_old);
        apply_dinv(M->nbr, M->br, dinv, r, t);
        #pragma omp parallel for schedule(static) if ((n) > OR_PAR_MIN)
        for (int i = 0; i < n; ++i) d[i] = rho_new * rho_old * d[i] + (2.0 * rho_new / delta) * t[i];
        rho_old = rho_new;
    }
    free(t);
}

static void vcycle(amg *H, int l);

/* K-cycle coarse solve on level c (Notay's Krylov-accelerated cycle): two
 * steps of GCR on L_c e = b_c, each preconditioned by one cycle on level c;
 * the result goes to x_c.  With w_1 = L_c z_1, a_1 = (w_1.b)/(w_1.w_1),
 * r_1 = b - a_1 w_1; w_2 = L_c z_2 - beta w_1, z_2 -= beta z_1 with
 * beta = (L_c z_2 . w_1)/(w_1.w_1); a_2 = (w_2.r_1)/(w_2.w_2);
 * e = a_1 z_1 + a_2 z_2. */
static void kcycle(amg *H, int c) {
    bmat *M = &H->L[c];
    int n = M->nbr * H->bs;
    double *b = H->bl[c], *r = H->kr[c], *z1 = H->kz1[c], *w1 = H->kw1[c], *z2 = H->kz2[c], *w2 = H->kw2[c];
    memcpy(r, b, sizeof(double) * n);
    vcycle(H, c);                                   /* z1 = cycle(b) */
    memcpy(z1, H->xl[c], sizeof(double) * n);
    spmv(M, z1, w1);
    double ww = dot(n, w1, w1);
    double a1 = (ww > 0.0) ? dot(n, w1, r) / ww : 0.0;
#pragma omp parallel for schedule(static) if ((n) > OR_PAR_MIN)
    for (int i = 0; i < n; ++i) r[i] = r[i] - a1 * w1[i];
    memcpy(b, r, sizeof(double) * n);               /* z2 = cycle(r_1) */
    vcycle(H, c);
    memcpy(z2, H->xl[c], sizeof(double) * n);
    spmv(M, z2, w2);
    double beta = (ww > 0.0) ? dot(n, w2, w1) / ww : 0.0;
#pragma omp parallel for schedule(static) if ((n) > OR_PAR_MIN)
    for (int i = 0; i < n; ++i) { w2[i] = w2[i] - beta * w1[i]; z2[i] = z2[i] - beta * z1[i]; }
    double w22 = dot(n, w2, w2);
    double a2 = (w22 > 0.0) ? dot(n, w2, r) / w22 : 0.0;
    double *x = H->xl[c];
#pragma omp parallel for schedule(static) if ((n) > OR_PAR_MIN)
    for (int i = 0; i < n; ++i) x[i] = a1 * z1[i] + a2 * z2[i];
}

/* V(1,1)-cycle on level l: x_l ~= L_l^{-1} b_l */
static void vcycle(amg *H, int l) {
    bmat *M = &H->L[l];
    int n = M->nbr * H->bs, bs = H->bs;
    double *b = H->bl[l], *x = H->xl[l], *r = H->rl[l], *d = H->dl[l];
    if (l == H->nlev - 1) { dense_lu_solve(H->nc, H->lu, H->piv, b, x); return; }
#pragma omp parallel for schedule(static) if ((n) > OR_PAR_MIN)
    for (int i = 0; i < n; ++i) x[i] = 0.0;
    chebyshev(M, H->dinv[l], H->rho[l], H->cheb_lo, H->cheb_degree, b, x, r, d, 1);
    double *t = dvec(n);
    spmv(M, x, t);
#pragma omp parallel for schedule(static) if ((n) > OR_PAR_MIN)
    for (int i = 0; i < n; ++i) r[i] = b[i] - t[i];
    int nc = H->L[l + 1].nbr;
    double *bc = H->bl[l + 1];
    const int *mp = H->mptr[l], *mb = H->mem[l];
#pragma omp parallel for schedule(static) if ((nc) > OR_PAR_MIN)
    for (int I = 0; I < nc; ++I)                  /* restriction P^T r: members in ascending i */
        for (int a = 0; a < bs; ++a) {
            double s = 0.0;
            for (int t = mp[I]; t < mp[I + 1]; ++t) s += r[(size_t)mb[t] * bs + a];
            bc[(size_t)I * bs + a] = s;
        }
    if (H->cycle == 1 && l + 1 < H->nlev - 1 && l + 1 <= H->kdepth) kcycle(H, l + 1);
    else vcycle(H, l + 1);
    const double *xc = H->xl[l + 1];
#pragma omp parallel for schedule(static) if ((M->nbr) > OR_PAR_MIN)
    for (int i = 0; i < M->nbr; ++i)              /* prolongation x += P e_c */
        if (H->agg[l][i] >= 0)
            for (int a = 0; a < bs; ++a) x[(size_t)i * bs + a] += xc[(size_t)H->agg[l][i] * bs + a];
    chebyshev(M, H->dinv[l], H->rho[l], H->cheb_lo, H->cheb_degree, b, x, r, d, 0);
    free(t);
}

static void amg_apply(amg *H, const double *b, double *x) {
    int n = H->L[0].nbr * H->bs;
    memcpy(H->bl[0], b, sizeof(double) * n);
    vcycle(H, 0);
    memcpy(x, H->xl[0], sizeof(double) * n);
}

/* ---------------------------------------------------------- S_hat */
/* diag(A) including the rank-one terms: A_ii + sum_k r_k (a^k_i)^2, k ascending */
static void diag_A(or_ctx *c) {
    int nv = 3 * c->N;
    free(c->diagA);
    c->diagA = dvec(nv);
    for (int i = 0; i < c->N; ++i) {
        int e = find_entry(&c->A, i, i);
        for (int a = 0; a < 3; ++a) c->diagA[3 * i + a] = (e >= 0) ? c->A.v[(size_t)e * 9 + 4 * a] : 0.0;
    }
    for (int k = 0; k < c->n_out; ++k)
        for (int e = c->out_ptr[k]; e < c->out_ptr[k + 1]; ++e) {
            double v = c->out_val[e];
            c->diagA[c->out_idx[e]] = c->diagA[c->out_idx[e]] + c->r[k] * (v * v);
        }
}

/* S_hat = D - C diag(A)^{-1} B (Sec. 3.1).  Entry (i,j): start from D_ij
 * (0 if absent) and subtract, for k ascending over row i of C, the term
 * t = (C_ik0 dinv_3k) B_kj0 + (C_ik1 dinv_3k+1) B_kj1 + (C_ik2 dinv_3k+2) B_kj2. */
static void build_shat(or_ctx *c) {
    int N = c->N;
    diag_A(c);
    double *dinv = dvec(3 * (size_t)N);
    for (int i = 0; i < 3 * N; ++i) dinv[i] = 1.0 / c->diagA[i];
    int *marker = (int *)xmalloc(sizeof(int) * N);
    for (int i = 0; i < N; ++i) marker[i] = -1;
    /* pass 1: count */
    long tot = 0;
    int *rp = (int *)xmalloc(sizeof(int) * (N + 1));
    for (int i = 0; i < N; ++i) {
        rp[i] = (int)tot;
        long start = tot;
        for (int e = c->D.rp[i]; e < c->D.rp[i + 1]; ++e) { int j = c->D.ci[e]; if (marker[j] < start) { marker[j] = (int)tot++; } }
        for (int e = c->C.rp[i]; e < c->C.rp[i + 1]; ++e) {
            int k = c->C.ci[e];
            for (int f = c->B.rp[k]; f < c->B.rp[k + 1]; ++f) { int j = c->B.ci[f]; if (marker[j] < start) { marker[j] = (int)tot++; } }
        }
    }
    rp[N] = (int)tot;
    for (int i = 0; i < N; ++i) marker[i] = -1;
    int *ci = (int *)xmalloc(sizeof(int) * (size_t)(tot + 1));
    double *v = (double *)xmalloc(sizeof(double) * (size_t)(tot + 1));
    for (int i = 0; i < N; ++i) {
        int pos = rp[i], start = rp[i];
        for (int e = c->D.rp[i]; e < c->D.rp[i + 1]; ++e) {
            int j = c->D.ci[e];
            if (marker[j] < start) { marker[j] = pos; ci[pos] = j; v[pos] = c->D.v[e]; ++pos; }
            else v[marker[j]] = v[marker[j]] + c->D.v[e];
        }
        for (int e = c->C.rp[i]; e < c->C.rp[i + 1]; ++e) {
            int k = c->C.ci[e];
            const double *cb = c->C.v + (size_t)e * 3;
            double w0 = cb[0] * dinv[3 * k], w1 = cb[1] * dinv[3 * k + 1], w2 = cb[2] * dinv[3 * k + 2];
            for (int f = c->B.rp[k]; f < c->B.rp[k + 1]; ++f) {
                int j = c->B.ci[f];
                const double *bb = c->B.v + (size_t)f * 3;
                double t = w0 * bb[0];
                t = t + w1 * bb[1];
                t = t + w2 * bb[2];
                if (marker[j] < start) { marker[j] = pos; ci[pos] = j; v[pos] = 0.0 - t; ++pos; }
                else v[marker[j]] = v[marker[j]] - t;
            }
        }
        /* sort row by column */
        for (int a = start + 1; a < pos; ++a) {
            int jj = ci[a]; double vv = v[a]; int b = a - 1;
            while (b >= start && ci[b] > jj) { ci[b + 1] = ci[b]; v[b + 1] = v[b]; --b; }
            ci[b + 1] = jj; v[b + 1] = vv;
        }
    }
    bmat_free(&c->Shat);
    c->Shat.nbr = N; c->Shat.nbc = N; c->Shat.br = 1; c->Shat.bc = 1;
    c->Shat.rp = rp; c->Shat.ci = ci; c->Shat.v = v;
    free(marker); free(dinv);
}

/* ---------------------------------------------------------- nested solve */
static void op_A(void *ctx, const double *x, double *y) { or_apply_A((or_ctx *)ctx, x, y); }
static void pc_A(void *ctx, const double *x, double *y) {
    or_ctx *c = (or_ctx *)ctx;
    if (c->opt.pc_A == 1) {
        const int n = 3 * c->N;
#pragma omp parallel for schedule(static) if ((n) > OR_PAR_MIN)
        for (int i = 0; i < n; ++i) y[i] = x[i] / c->diagA[i];
        return;
    }
    amg_apply(&c->amgA, x, y);
}
static void pc_S(void *ctx, const double *x, double *y) {
    or_ctx *c = (or_ctx *)ctx;
    if (c->opt.pc_S == 1) { memcpy(y, x, sizeof(double) * c->N); return; }
    amg_apply(&c->amgS, x, y);
}

/* GMRES(m_A) + P_A on A y = s to relative tolerance rtol (Sec. 3.1) */
int or_solve_A(or_ctx *c, const double *s, double *y, double rtol, int *its) {
    double rel;
    int rc = fgmres(3 * c->N, op_A, c, pc_A, c, s, y, rtol, c->opt.atol, c->opt.m_A, c->opt.nmax_A, 0, its, &rel, NULL);
    return rc;
}

/* Algorithm 2: S x_p = D x_p - C A^{-1} B x_p, inner solve with delta_I */
void or_apply_S(or_ctx *c, const double *xp, double *y) {
    int N = c->N, its;
    double *xhat = dvec(N), *xbar = dvec(3 * (size_t)N), *xtil = dvec(3 * (size_t)N), *cx = dvec(N);
    spmv(&c->D, xp, xhat);                                 /* line 1 */
    spmv(&c->B, xp, xbar);                                 /* line 2 */
    const int deg = c->amgA.cheb_degree;                   /* line 3, with its own cycle degree */
    c->amgA.cheb_degree = c->opt.cheb_degree_I;
    or_solve_A(c, xbar, xtil, c->opt.rtol_I, &its);
    c->amgA.cheb_degree = deg;
    c->info.I_iters += its; c->info.n_I_solves++;
    spmv(&c->C, xtil, cx);                                 /* line 4 */
#pragma omp parallel for schedule(static) if ((N) > OR_PAR_MIN)
    for (int i = 0; i < N; ++i) y[i] = xhat[i] - cx[i];    /* line 5 */
    free(xhat); free(xbar); free(xtil); free(cx);
}
static void op_S(void *ctx, const double *x, double *y) { or_apply_S((or_ctx *)ctx, x, y); }

static void op_Shat(void *ctx, const double *x, double *y) { spmv(&((or_ctx *)ctx)->Shat, x, y); }

/* SIMPLE (Sec. 3.2): P = [[I,0],[C A^{-1},I]] [[A,0],[0,S_hat]] [[I, diag(A)^{-1} B],[0,I]];
 * its inverse is Algorithm 3 with steps 3-4 replaced by a GMRES(m_S) solve with
 * S_hat (P_S = AMG(S_hat)) and y_v = y_hat_v - diag(A)^{-1} B y_p, no step 5. */
static void apply_simple(or_ctx *c, const double *s, double *y) {
    int N = c->N, nv = 3 * N, its;
    double rel;
    double *sp2 = dvec(N), *t = dvec(nv), *ct = dvec(N);
    or_solve_A(c, s, y, c->opt.rtol_A, &its);                                /* step 1 */
    c->info.A_iters += its; c->info.n_A_solves++;
    spmv(&c->C, y, ct);                                                       /* step 2 */
    for (int i = 0; i < N; ++i) sp2[i] = s[nv + i] - ct[i];
    fgmres(N, op_Shat, c, pc_S, c, sp2, y + nv, c->opt.rtol_S, c->opt.atol, c->opt.m_S, c->opt.nmax_S, 0, &its, &rel,
           NULL);                                                             /* step 3' */
    c->info.S_iters += its; c->info.n_S_solves++;
    spmv(&c->B, y + nv, t);                                                   /* step 4' */
    for (int i = 0; i < nv; ++i) y[i] = y[i] - t[i] / c->diagA[i];
    free(sp2); free(t); free(ct);
}

/* Algorithm 3: y = P_SCR^{-1} s (variant 1: upper block-triangular [[A,B],[0,S]];
 * variant 2: SIMPLE) */
void or_apply_pscr(or_ctx *c, const double *s, double *y) {
    if (c->opt.variant == 2) { apply_simple(c, s, y); return; }
    int N = c->N, nv = 3 * N, its;
    double rel;
    const double *sv = s, *sp = s + nv;
    double *yv = y, *yp = y + nv;
    double *sp2 = dvec(N), *sv2 = dvec(nv), *t = dvec(nv);
    memcpy(sp2, sp, sizeof(double) * N);
    if (c->opt.variant == 0) {
        or_solve_A(c, sv, t, c->opt.rtol_A, &its);                 /* step 1 */
        c->info.A_iters += its; c->info.n_A_solves++;
        double *ct = dvec(N);
        spmv(&c->C, t, ct);                                        /* step 2 */
        for (int i = 0; i < N; ++i) sp2[i] = sp2[i] - ct[i];
        free(ct);
    }
    fgmres(N, op_S, c, pc_S, c, sp2, yp, c->opt.rtol_S, c->opt.atol, c->opt.m_S, c->opt.nmax_S, 0, &its, &rel, NULL); /* step 3 */
    c->info.S_iters += its; c->info.n_S_solves++;
    spmv(&c->B, yp, t);                                            /* step 4 */
#pragma omp parallel for schedule(static) if ((nv) > OR_PAR_MIN)
    for (int i = 0; i < nv; ++i) sv2[i] = sv[i] - t[i];
    or_solve_A(c, sv2, yv, c->opt.rtol_A, &its);                   /* step 5 */
    c->info.A_iters += its; c->info.n_A_solves++;
    free(sp2); free(sv2); free(t);
}

static void op_full(void *ctx, const double *x, double *y) { or_apply_full((or_ctx *)ctx, x, y); }
static void pc_scr(void *ctx, const double *x, double *y) { or_apply_pscr((or_ctx *)ctx, x, y); }

/* Outer FGMRES(m) with P_SCR (Sec. 3): x = A^{-1} b to delta^r */
int or_solve(or_ctx *c, const double *b, double *x, or_info *info) {
    memset(&c->info, 0, sizeof(c->info));
    int its;
    double rel, relt;
    int rc = fgmres(4 * c->N, op_full, c, pc_scr, c, b, x, c->opt.rtol, c->opt.atol, c->opt.m, c->opt.nmax, 1, &its, &rel,
                    &relt);
    c->info.outer_iters = its;
    c->info.rel_res_est = rel;
    c->info.rel_res_true = relt;
    c->info.status = rc;
    if (info) *info = c->info;
    return rc;
}

/* --------------------------------------------------------------- context */
void or_default_options(or_options *o) {
    o->rtol = 1e-8; o->rtol_A = 1e-3; o->rtol_S = 1e-2; o->rtol_I = 1e-2; o->atol = 1e-50;
    o->m = 200; o->m_A = 200; o->m_S = 200; o->nmax = 200; o->nmax_A = 200; o->nmax_S = 200;
    o->pc_A = 0; o->pc_S = 0; o->variant = 0;
    o->amg_max_levels = 5; o->amg_coarse_max = 300; o->cheb_degree = 2; o->theta = 0.0064;
    o->amg_cycle = 1;
    o->amg_kdepth = 2;
    o->cheb_degree_S = 1;
    o->cheb_degree_I = 1;
}

or_ctx *or_create(int N, const int *arp, const int *aci, const double *av, const int *brp, const int *bci,
                  const double *bv, const int *crp, const int *cci, const double *cv, const int *drp, const int *dci,
                  const double *dv, int n_out, const int *optr, const int *oidx, const double *oval, const double *r) {
    or_ctx *c = (or_ctx *)calloc(1, sizeof(or_ctx));
    c->N = N;
    bmat_copy(&c->A, N, N, 3, 3, arp, aci, av);
    bmat_copy(&c->B, N, N, 3, 1, brp, bci, bv);
    bmat_copy(&c->C, N, N, 1, 3, crp, cci, cv);
    bmat_copy(&c->D, N, N, 1, 1, drp, dci, dv);
    c->n_out = n_out;
    int no = n_out > 0 ? optr[n_out] : 0;
    c->out_ptr = (int *)xmalloc(sizeof(int) * (n_out + 1));
    c->out_idx = (int *)xmalloc(sizeof(int) * (no + 1));
    c->out_val = dvec(no + 1);
    c->r = dvec(n_out + 1);
    if (n_out > 0) {
        memcpy(c->out_ptr, optr, sizeof(int) * (n_out + 1));
        memcpy(c->out_idx, oidx, sizeof(int) * no);
        memcpy(c->out_val, oval, sizeof(double) * no);
        memcpy(c->r, r, sizeof(double) * n_out);
    } else c->out_ptr[0] = 0;
    c->wv1 = dvec(3 * (size_t)N); c->wv2 = dvec(3 * (size_t)N); c->wv3 = dvec(3 * (size_t)N);
    c->wp1 = dvec(N); c->wp2 = dvec(N); c->wp3 = dvec(N); c->wp4 = dvec(N);
    or_default_options(&c->opt);
    diag_A(c);
    return c;
}

/* New operator values on the same patterns (a later Newton tangent, Sec.
 * 2.5); the preconditioner built by the last or_setup -- AMG(A), S_hat,
 * AMG(S_hat) -- is kept, which makes it a lagged preconditioner of the new
 * operator (the outer FGMRES accepts any preconditioner, Sec. 3). */
void or_set_values(or_ctx *c, const double *av, const double *bv, const double *cv, const double *dv) {
    memcpy(c->A.v, av, sizeof(double) * (size_t)c->A.rp[c->N] * 9);
    memcpy(c->B.v, bv, sizeof(double) * (size_t)c->B.rp[c->N] * 3);
    memcpy(c->C.v, cv, sizeof(double) * (size_t)c->C.rp[c->N] * 3);
    memcpy(c->D.v, dv, sizeof(double) * (size_t)c->D.rp[c->N]);
}

/* Threads of the parallel loops (timing only: results are the same at any
 * count); n <= 0 leaves the count unchanged.  Returns the count in use. */
int or_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

void or_set_options(or_ctx *c, const or_options *o) { c->opt = *o; }
void or_get_options(const or_ctx *c, or_options *o) { *o = c->opt; }

void or_set_resistances(or_ctx *c, const double *r) {
    if (c->n_out > 0) memcpy(c->r, r, sizeof(double) * c->n_out);
    diag_A(c);
}

/* AMG(A_sp), S_hat and AMG(S_hat) */
int or_setup(or_ctx *c) {
    if (c->have_amgA) amg_free(&c->amgA);
    if (c->have_amgS) amg_free(&c->amgS);
    amg_build(&c->amgA, &c->A, &c->opt, c->opt.amg_cycle == 2, c->opt.cheb_degree, 1, 10.0, NULL);
    c->have_amgA = 1;
    build_shat(c);
    amg_build(&c->amgS, &c->Shat, &c->opt, c->opt.amg_cycle >= 1, c->opt.cheb_degree_S, 0, 3.0, NULL);
    c->have_amgS = 1;
    return 0;
}

/* Numeric re-setup after new values on the same patterns (a later Newton
 * tangent, Sec. 2.5): AMG(A), S_hat and AMG(S_hat) rebuilt from the current
 * values on the aggregates of the last or_setup -- Galerkin operators,
 * block-diagonal inverses, Chebyshev bounds and coarsest factorisations all
 * new, only the aggregation is kept.  Returns 1 without a previous setup. */
int or_setup_numeric(or_ctx *c) {
    if (!c->have_amgA || !c->have_amgS) return 1;
    amg oldA = c->amgA, oldS = c->amgS;
    amg_build(&c->amgA, &c->A, &c->opt, c->opt.amg_cycle == 2, c->opt.cheb_degree, 1, 10.0, &oldA);
    amg_free(&oldA);
    build_shat(c);
    amg_build(&c->amgS, &c->Shat, &c->opt, c->opt.amg_cycle >= 1, c->opt.cheb_degree_S, 0, 3.0, &oldS);
    amg_free(&oldS);
    return 0;
}

void or_vcycle(or_ctx *c, int which, const double *b, double *x) { amg_apply(which ? &c->amgS : &c->amgA, b, x); }

/* The same cycle with Chebyshev degree `degree` (the inner A-solves' cycle of
 * Algorithm 2 when degree = cheb_degree_I) */
void or_vcycle_degree(or_ctx *c, int which, int degree, const double *b, double *x) {
    amg *H = which ? &c->amgS : &c->amgA;
    const int keep = H->cheb_degree;
    H->cheb_degree = degree;
    amg_apply(H, b, x);
    H->cheb_degree = keep;
}

int or_amg_nlev(or_ctx *c, int which) { return (which ? &c->amgS : &c->amgA)->nlev; }
int or_amg_level_rows(or_ctx *c, int which, int l) { return (which ? &c->amgS : &c->amgA)->L[l].nbr; }
int or_amg_level_nnz(or_ctx *c, int which, int l) { amg *H = which ? &c->amgS : &c->amgA; return H->L[l].rp[H->L[l].nbr]; }
double or_amg_level_rho(or_ctx *c, int which, int l) { return (which ? &c->amgS : &c->amgA)->rho[l]; }
void or_amg_level_get(or_ctx *c, int which, int l, int *rp, int *ci, double *v, int *agg) {
    amg *H = which ? &c->amgS : &c->amgA;
    bmat *M = &H->L[l];
    int nb = M->br * M->bc, nnz = M->rp[M->nbr];
    if (rp) memcpy(rp, M->rp, sizeof(int) * (M->nbr + 1));
    if (ci) memcpy(ci, M->ci, sizeof(int) * nnz);
    if (v) memcpy(v, M->v, sizeof(double) * (size_t)nnz * nb);
    if (agg && H->agg[l]) memcpy(agg, H->agg[l], sizeof(int) * M->nbr);
}
int or_shat_nnz(or_ctx *c) { return c->Shat.rp ? c->Shat.rp[c->N] : 0; }
void or_shat_get(or_ctx *c, int *rp, int *ci, double *v) {
    int nnz = c->Shat.rp[c->N];
    memcpy(rp, c->Shat.rp, sizeof(int) * (c->N + 1));
    memcpy(ci, c->Shat.ci, sizeof(int) * nnz);
    memcpy(v, c->Shat.v, sizeof(double) * nnz);
}
void or_diag_A(or_ctx *c, double *out) { memcpy(out, c->diagA, sizeof(double) * 3 * c->N); }

/* strength weights and one matching pass, exposed for pin tests */
int or_strength_and_aggregate(int nbr, int bs, const int *rp, const int *ci, const double *v, double theta, int *agg) {
    bmat M = {nbr, nbr, bs, bs, (int *)rp, (int *)ci, (double *)v};
    return aggregate(&M, theta, agg);
}

/* Chebyshev smoother, exposed for pin tests: x <- smoothed x (x in/out) */
void or_chebyshev(int nbr, int bs, const int *rp, const int *ci, const double *v, double rho, double lodiv, int k,
                  const double *b, double *x, int x_is_zero) {
    bmat M = {nbr, nbr, bs, bs, (int *)rp, (int *)ci, (double *)v};
    int n = nbr * bs;
    double *dinv = dvec((size_t)nbr * bs * bs), *r = dvec(n), *d = dvec(n);
    block_diag_inv(&M, dinv);
    chebyshev(&M, dinv, rho, lodiv, k, b, x, r, d, x_is_zero);
    free(dinv); free(r); free(d);
}

/* generic GMRES on A (without preconditioner or with P_A), exposed for pin tests */
int or_gmres_A(or_ctx *c, const double *b, double *x, double rtol, int m, int nmax, int use_pc, int *its, double *rel) {
    return fgmres(3 * c->N, op_A, c, use_pc ? pc_A : NULL, c, b, x, rtol, c->opt.atol, m, nmax, 0, its, rel, NULL);
}

void or_get_info(const or_ctx *c, or_info *info) { *info = c->info; }

void or_destroy(or_ctx *c) {
    if (!c) return;
    bmat_free(&c->A); bmat_free(&c->B); bmat_free(&c->C); bmat_free(&c->D); bmat_free(&c->Shat);
    if (c->have_amgA) amg_free(&c->amgA);
    if (c->have_amgS) amg_free(&c->amgS);
    free(c->out_ptr); free(c->out_idx); free(c->out_val); free(c->r); free(c->diagA);
    free(c->wv1); free(c->wv2); free(c->wv3); free(c->wp1); free(c->wp2); free(c->wp3); free(c->wp4);
    free(c);
}

/* ------------------------------------------------------------ RCR outlets */
/* right-hand side of the distal-pressure ODE (Sec. 2.1, RCR circuit) */
static double rcr_rhs(double Pi, double Q, double Rd, double C) { return -Pi / (Rd * C) + Q / C; }

/* Algorithm 1: Pi over [t_n, t_n + dt] in n_ts equal substeps h, Q linear
 * from Q_n to Q_np1 (Q_{n,m} = (1 - m/n_ts) Q_n + (m/n_ts) Q_np1); stages
 * K1..K4 with the intermediate flows 2/3 Q_m + 1/3 Q_{m+1} and
 * 1/3 Q_m + 2/3 Q_{m+1}; weights 1/8, 3/8, 3/8, 1/8.  Returns
 * P_{n+1} = R_p Q_np1 + Pi_{n,n_ts} + P_d and the end value of Pi. */
static double rcr_G(double Rp, double C, double Rd, double Pd, double Pi_n, double Q_n, double Q_np1, double dt,
                    int nts, double *Pi_end) {
    const double h = dt / nts;
    double Pi = Pi_n;
    for (int m = 0; m < nts; ++m) {
        const double Qa = (1.0 - (double)m / nts) * Q_n + ((double)m / nts) * Q_np1;
        const double Qb = (1.0 - (double)(m + 1) / nts) * Q_n + ((double)(m + 1) / nts) * Q_np1;
        const double K1 = rcr_rhs(Pi, Qa, Rd, C);
        const double K2 = rcr_rhs(Pi + K1 * h / 3.0, 2.0 * Qa / 3.0 + Qb / 3.0, Rd, C);
        const double K3 = rcr_rhs(Pi - K1 * h / 3.0 + K2 * h, Qa / 3.0 + 2.0 * Qb / 3.0, Rd, C);
        const double K4 = rcr_rhs(Pi + K1 * h - K2 * h + K3 * h, Qb, Rd, C);
        Pi = Pi + K1 * h / 8.0 + 3.0 * K2 * h / 8.0 + 3.0 * K3 * h / 8.0 + K4 * h / 8.0;
    }
    if (Pi_end) *Pi_end = Pi;
    return Rp * Q_np1 + Pi + Pd;
}

/* One step for n_out outlets: P_np1 = G(Pi_n, Q_n, Q_np1), Pi_np1 its end
 * state, and m = (G(.., Q_np1 + eps/2) - G(.., Q_np1 - eps/2)) / eps with
 * eps = max(eps_abs, eps_rel |Q_np1|) (Sec. 2.5, difference approximation
 * of m^k). */
void or_rcr_step(int n_out, const double *Rp, const double *C, const double *Rd, const double *Pd, const double *Pi_n,
                 const double *Q_n, const double *Q_np1, double dt, int nts, double eps_abs, double eps_rel,
                 double *P_np1, double *Pi_np1, double *m) {
    for (int k = 0; k < n_out; ++k) {
        P_np1[k] = rcr_G(Rp[k], C[k], Rd[k], Pd[k], Pi_n[k], Q_n[k], Q_np1[k], dt, nts, &Pi_np1[k]);
        const double eps = fmax(eps_abs, eps_rel * fabs(Q_np1[k]));
        const double Pp = rcr_G(Rp[k], C[k], Rd[k], Pd[k], Pi_n[k], Q_n[k], Q_np1[k] + eps / 2.0, dt, nts, NULL);
        const double Pm = rcr_G(Rp[k], C[k], Rd[k], Pd[k], Pi_n[k], Q_n[k], Q_np1[k] - eps / 2.0, dt, nts, NULL);
        m[k] = (Pp - Pm) / eps;
    }
}
