/*
 * synth.c -- seeded synthetic inputs for the nested block solve.
 *
 * This module produces INPUT DATA only: a hex-to-tet box mesh, the P1-P1
 * residual-based VMS / generalized-alpha consistent tangent [[A,B],[C,D]]
 * linearised about a seeded perturbed Poiseuille state, the outlet vectors
 * a^k and the right-hand side.  It holds none of the solver's arithmetic and
 * is shared, as a data source, by the oracle and by the CUDA path.
 *
 * Discretisation followed (paper Sec. 2.3-2.5):
 *   - momentum residual B_m^vol (Eq. for B_m^vol, Sec. 2.3), backflow term
 *     B_m^bf (beta = 0.2), continuity residual B_p, fine scales
 *     v' = -tau_M r_M, p' = -tau_C div v, tau_M / tau_C / G / M as in Sec. 2.3
 *     with C_I = 36, C_T = 4;
 *   - tangent blocks A = alpha_m dR_m/dvdot + alpha_f gamma dt dR_m/dv
 *     (+ backflow), B = alpha_f gamma dt dR_m/dp, C = alpha_m dR_p/dvdot +
 *     alpha_f gamma dt dR_p/dv, D = alpha_f gamma dt dR_p/dp (Sec. 2.5,
 *     definitions of A, B, C, D); the resistance part K is NOT assembled: it is
 *     returned as the outlet vectors a^k_{Ai} = int_{Gamma_k} N_A n_i and
 *     applied matrix-free by the solvers;
 *   - generalized-alpha parameters from rho_inf (Sec. 2.4.1).
 * Reading taken where the paper is silent: tau_M, tau_C (and G) are frozen at
 * the linearisation state; everything else is differentiated exactly.  The
 * linearisation state has vdot = 0, p = 0, body force 0.  Dirichlet velocity
 * dofs (walls x,y in {0,L}, inlet z = 0) keep their assembled diagonal entry
 * and get zero off-diagonal A entries in their row and column, zero B rows and
 * zero C columns (the sparsity pattern keeps the explicit zeros).
 *
 * Mesh: nx*ny*nz hexes, each split into the 6 Kuhn tetrahedra sharing the
 * (0,0,0)-(1,1,1) diagonal; nodes numbered x fastest, then y, then z.  Every
 * interior node has 14 neighbours (15 blocks per row).  A, B, C, D share one
 * node-graph pattern (rowptr, col) with 9, 3, 3, 1 values per entry
 * (row-major 3x3 blocks for A; B block = column 3-vector, C block = row
 * 3-vector).
 *
 * Random numbers: SplitMix64 (Steele, Lea & Flood 2014), u = (x >> 11) 2^-53.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int nx, ny, nz;
    double Lx, Ly, Lz;
    double Re, rho, mu, dt, rho_inf;
    double pert;      /* relative perturbation amplitude (0.05) */
    uint64_t seed;
    int n_out;        /* outlet pieces on the z = Lz face: 1..4 (halves, thirds,
                         quadrants) or up to 2 nx ny patches of consecutive triangles */
} synth_params;

static inline uint64_t sm64_next(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static inline double sm64_u01(uint64_t *s) { return (double)(sm64_next(s) >> 11) * 0x1.0p-53; }

/* ------------------------------------------------------------------ mesh */
static inline long nid(const synth_params *p, int i, int j, int k) {
    return (long)i + (long)(p->nx + 1) * ((long)j + (long)(p->ny + 1) * (long)k);
}

/* The 14 Kuhn-split neighbour offsets plus self, sorted by index delta. */
static void neighbour_offsets(const synth_params *p, int off[15][3]) {
    int cnt = 0;
    long keys[15];
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int pos = (dx > 0) || (dy > 0) || (dz > 0);
                int neg = (dx < 0) || (dy < 0) || (dz < 0);
                if (pos && neg) continue;
                off[cnt][0] = dx; off[cnt][1] = dy; off[cnt][2] = dz;
                keys[cnt] = dx + (long)(p->nx + 1) * (dy + (long)(p->ny + 1) * dz);
                cnt++;
            }
    /* insertion sort by key (keys are distinct) */
    for (int a = 1; a < 15; ++a) {
        long k = keys[a]; int o0 = off[a][0], o1 = off[a][1], o2 = off[a][2];
        int b = a - 1;
        while (b >= 0 && keys[b] > k) {
            keys[b + 1] = keys[b];
            off[b + 1][0] = off[b][0]; off[b + 1][1] = off[b][1]; off[b + 1][2] = off[b][2];
            --b;
        }
        keys[b + 1] = k; off[b + 1][0] = o0; off[b + 1][1] = o1; off[b + 1][2] = o2;
    }
}

static inline int in_range(const synth_params *p, int i, int j, int k) {
    return i >= 0 && j >= 0 && k >= 0 && i <= p->nx && j <= p->ny && k <= p->nz;
}

static inline int is_dirichlet(const synth_params *p, int i, int j, int k) {
    return i == 0 || i == p->nx || j == 0 || j == p->ny || k == 0;
}

/* Kuhn tetrahedron t (0..5) of the unit hex: corner codes bx + 2 by + 4 bz. */
static void kuhn_tet(int t, int c[4]) {
    static const int perm[6][3] = {{0,1,2},{0,2,1},{1,0,2},{1,2,0},{2,0,1},{2,1,0}};
    c[0] = 0;
    c[1] = 1 << perm[t][0];
    c[2] = c[1] | (1 << perm[t][1]);
    c[3] = 7;
}

long synth_num_nodes(const synth_params *p) {
    return (long)(p->nx + 1) * (p->ny + 1) * (p->nz + 1);
}

/* Row pointer of the shared node-graph pattern; returns nnz. */
long synth_pattern(const synth_params *p, int32_t *rowptr, int32_t *col) {
    int off[15][3];
    neighbour_offsets(p, off);
    long n = 0;
    long N = synth_num_nodes(p);
    for (int k = 0; k <= p->nz; ++k)
        for (int j = 0; j <= p->ny; ++j)
            for (int i = 0; i <= p->nx; ++i) {
                long a = nid(p, i, j, k);
                if (rowptr) rowptr[a] = (int32_t)n;
                for (int q = 0; q < 15; ++q) {
                    int ii = i + off[q][0], jj = j + off[q][1], kk = k + off[q][2];
                    if (!in_range(p, ii, jj, kk)) continue;
                    if (col) col[n] = (int32_t)nid(p, ii, jj, kk);
                    ++n;
                }
            }
    if (rowptr) rowptr[N] = (int32_t)n;
    return n;
}

/* --------------------------------------------------- linearisation state */
/* Nodal velocity: 16 U x(1-x) y(1-y) e_z (box width as the length scale, x,y
 * scaled to [0,1]) plus a per-component uniform +-pert*U perturbation at
 * non-Dirichlet nodes; Dirichlet nodes keep the base profile (zero on walls,
 * Poiseuille on the inlet).  Draw order: node index ascending, components
 * x,y,z, one draw each for every node (Dirichlet draws are discarded). */
void synth_state(const synth_params *p, double *vel /* 3N */) {
    uint64_t s = p->seed;
    double U = p->Re * p->mu / (p->rho * p->Lx);
    for (int k = 0; k <= p->nz; ++k)
        for (int j = 0; j <= p->ny; ++j)
            for (int i = 0; i <= p->nx; ++i) {
                long a = nid(p, i, j, k);
                double x = (double)i / p->nx, y = (double)j / p->ny;
                double base[3] = {0.0, 0.0, 16.0 * U * x * (1.0 - x) * y * (1.0 - y)};
                int dir = is_dirichlet(p, i, j, k);
                for (int c = 0; c < 3; ++c) {
                    double u = sm64_u01(&s);
                    vel[3 * a + c] = base[c] + (dir ? 0.0 : p->pert * U * (2.0 * u - 1.0));
                }
            }
}

/* ----------------------------------------------------- element kernels */
typedef struct {
    double am, c;              /* alpha_m, alpha_f*gamma*dt */
    double rho, mu, dt;
} coefs;

static void gen_alpha(const synth_params *p, coefs *cf) {
    double ri = p->rho_inf;
    double am = 0.5 * (3.0 - ri) / (1.0 + ri);
    double af = 1.0 / (1.0 + ri), gm = 1.0 / (1.0 + ri);
    cf->am = am; cf->c = af * gm * p->dt; cf->rho = p->rho; cf->mu = p->mu; cf->dt = p->dt;
}

/* Shape-function gradients (rows) and volume of the tet with vertices X. */
static double tet_grads(const double X[4][3], double dN[4][3]) {
    double J[3][3];
    for (int r = 0; r < 3; ++r)
        for (int e = 0; e < 3; ++e) J[r][e] = X[e + 1][r] - X[0][r]; /* column e = edge e */
    double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
               - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
               + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    double inv[3][3];
    inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    /* xi_e = N_{e+1}; d xi_e / d x_r = inv[e][r] */
    for (int r = 0; r < 3; ++r) {
        dN[1][r] = inv[0][r]; dN[2][r] = inv[1][r]; dN[3][r] = inv[2][r];
        dN[0][r] = -(inv[0][r] + inv[1][r] + inv[2][r]);
    }
    return fabs(det) / 6.0;
}

/* Contributions of one tet to the rows of local node `la`:
 * Ab[lb][i][j] (3x3), Bb[lb][i], Cb[lb][j], Db[lb] for lb = 0..3.
 * vel: the 4 nodal linearisation velocities. */
static void tet_rows(const coefs *cf, const double X[4][3], const double vel[4][3], int la,
                     double Ab[4][3][3], double Bb[4][3], double Cb[4][3], double Db[4]) {
    static const double qa = 0.5854101966249685, qb = 0.1381966011250105;
    const double CI = 36.0, CT = 4.0;
    double dN[4][3];
    double vol = tet_grads(X, dN);
    const double rho = cf->rho, mu = cf->mu;
    /* metric G_ij = sum_kl dxi_k/dx_i M_kl dxi_l/dx_j, M = 2^(1/3)/2 [[2,1,1],[1,2,1],[1,1,2]] */
    double Mm[3][3], m0 = 1.2599210498948732 / 2.0; /* 2^(1/3) / 2 */
    for (int r = 0; r < 3; ++r)
        for (int s = 0; s < 3; ++s) Mm[r][s] = m0 * (r == s ? 2.0 : 1.0);
    double G[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double g = 0.0;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) g += dN[k + 1][i] * Mm[k][l] * dN[l + 1][j];
            G[i][j] = g;
        }
    double GG = 0.0, trG = G[0][0] + G[1][1] + G[2][2];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) GG += G[i][j] * G[i][j];
    /* velocity gradient Ga_ij = d a_i / d x_j (constant) */
    double Ga[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double g = 0.0;
            for (int b = 0; b < 4; ++b) g += vel[b][i] * dN[b][j];
            Ga[i][j] = g;
        }
    memset(Ab, 0, sizeof(double) * 36); memset(Bb, 0, sizeof(double) * 12);
    memset(Cb, 0, sizeof(double) * 12); memset(Db, 0, sizeof(double) * 4);
    for (int q = 0; q < 4; ++q) {
        double N[4];
        for (int b = 0; b < 4; ++b) N[b] = (b == q) ? qa : qb;
        double w = vol / 4.0;
        double a[3] = {0, 0, 0};
        for (int b = 0; b < 4; ++b)
            for (int i = 0; i < 3; ++i) a[i] += N[b] * vel[b][i];
        double aGa = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) aGa += a[i] * G[i][j] * a[j];
        double tauM = 1.0 / (rho * sqrt(CT / (cf->dt * cf->dt) + aGa + CI * (mu / rho) * (mu / rho) * GG));
        double tauC = 1.0 / (tauM * trG);
        double vp[3]; /* v' = -tauM rho (a . grad) a */
        for (int i = 0; i < 3; ++i) {
            double s = 0.0;
            for (int j = 0; j < 3; ++j) s += Ga[i][j] * a[j];
            vp[i] = -tauM * rho * s;
        }
        const double *dNa = dN[la];
        double Na = N[la];
        double adNa = a[0] * dNa[0] + a[1] * dNa[1] + a[2] * dNa[2];
        double vpdNa = vp[0] * dNa[0] + vp[1] * dNa[1] + vp[2] * dNa[2];
        /* momentum row sensitivity to dv'_k */
        double Kvp[3][3];
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k)
                Kvp[i][k] = (i == k ? -rho * adNa - rho * vpdNa : 0.0) + rho * Na * Ga[i][k] - rho * vp[i] * dNa[k];
        for (int lb = 0; lb < 4; ++lb) {
            const double *dNb = dN[lb];
            double Nb = N[lb];
            double adNb = a[0] * dNb[0] + a[1] * dNb[1] + a[2] * dNb[2];
            double vpdNb = vp[0] * dNb[0] + vp[1] * dNb[1] + vp[2] * dNb[2];
            double dadb = dNa[0] * dNb[0] + dNa[1] * dNb[1] + dNa[2] * dNb[2];
            /* dv'/d(unknowns of node b) */
            double Pd[3][3], Pv[3][3], Pp[3];
            for (int k = 0; k < 3; ++k) {
                for (int j = 0; j < 3; ++j) {
                    Pd[k][j] = (k == j) ? -tauM * rho * Nb : 0.0;
                    Pv[k][j] = -tauM * rho * (Nb * Ga[k][j] + (k == j ? adNb : 0.0));
                }
                Pp[k] = -tauM * dNb[k];
            }
            for (int i = 0; i < 3; ++i) {
                for (int j = 0; j < 3; ++j) {
                    double dij = (i == j) ? 1.0 : 0.0;
                    double md = rho * Na * Nb * dij;
                    double kv = rho * Na * (Nb * Ga[i][j] + adNb * dij)
                              + mu * (dadb * dij + dNa[j] * dNb[i])
                              - rho * Nb * dNa[j] * vp[i]
                              + rho * Na * vpdNb * dij
                              + tauC * dNa[i] * dNb[j];
                    for (int k = 0; k < 3; ++k) {
                        md += Kvp[i][k] * Pd[k][j];
                        kv += Kvp[i][k] * Pv[k][j];
                    }
                    Ab[lb][i][j] += w * (cf->am * md + cf->c * kv);
                }
                double kp = -dNa[i] * Nb;
                for (int k = 0; k < 3; ++k) kp += Kvp[i][k] * Pp[k];
                Bb[lb][i] += w * cf->c * kp;
            }
            for (int j = 0; j < 3; ++j) {
                double cd = tauM * rho * Nb * dNa[j];
                double cv = Na * dNb[j] + tauM * rho * adNb * dNa[j];
                for (int k = 0; k < 3; ++k) cv += tauM * rho * dNa[k] * Nb * Ga[k][j];
                Cb[lb][j] += w * (cf->am * cd + cf->c * cv);
            }
            Db[lb] += w * cf->c * tauM * dadb;
        }
    }
}

/* Backflow contribution (B_m^bf, beta = 0.2, n = +e_z) of one outlet triangle
 * to the rows of local vertex `la` (A blocks only). */
static void tri_backflow_rows(const coefs *cf, const double X[3][3], const double vel[3][3], int la,
                              double Ab[3][3][3]) {
    const double beta = 0.2;
    double e1[3], e2[3], cr[3];
    for (int r = 0; r < 3; ++r) { e1[r] = X[1][r] - X[0][r]; e2[r] = X[2][r] - X[0][r]; }
    cr[0] = e1[1] * e2[2] - e1[2] * e2[1];
    cr[1] = e1[2] * e2[0] - e1[0] * e2[2];
    cr[2] = e1[0] * e2[1] - e1[1] * e2[0];
    double area = 0.5 * sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    const double n[3] = {0.0, 0.0, 1.0};
    memset(Ab, 0, sizeof(double) * 27);
    for (int q = 0; q < 3; ++q) {
        double N[3];
        for (int b = 0; b < 3; ++b) N[b] = (b == q) ? 2.0 / 3.0 : 1.0 / 6.0;
        double w = area / 3.0;
        double a[3] = {0, 0, 0};
        for (int b = 0; b < 3; ++b)
            for (int i = 0; i < 3; ++i) a[i] += N[b] * vel[b][i];
        double an = a[0] * n[0] + a[1] * n[1] + a[2] * n[2];
        if (!(an < 0.0)) continue;
        for (int lb = 0; lb < 3; ++lb)
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    Ab[lb][i][j] += w * cf->c * (-cf->rho * beta * N[la] * N[lb] * (n[j] * a[i] + (i == j ? an : 0.0)));
    }
}

/* Debug/test entry: the full 16x16 element tangent of one tet, ordered
 * (node a, dof d) with d = 0,1,2 velocity, 3 pressure. */
void synth_element_tangent(const synth_params *p, const double *X12, const double *vel12, double *K256) {
    coefs cf; gen_alpha(p, &cf);
    double X[4][3], vel[4][3];
    for (int a = 0; a < 4; ++a)
        for (int r = 0; r < 3; ++r) { X[a][r] = X12[3 * a + r]; vel[a][r] = vel12[3 * a + r]; }
    for (int la = 0; la < 4; ++la) {
        double Ab[4][3][3], Bb[4][3], Cb[4][3], Db[4];
        tet_rows(&cf, X, vel, la, Ab, Bb, Cb, Db);
        for (int lb = 0; lb < 4; ++lb) {
            for (int i = 0; i < 3; ++i) {
                for (int j = 0; j < 3; ++j) K256[(4 * la + i) * 16 + 4 * lb + j] = Ab[lb][i][j];
                K256[(4 * la + i) * 16 + 4 * lb + 3] = Bb[lb][i];
            }
            for (int j = 0; j < 3; ++j) K256[(4 * la + 3) * 16 + 4 * lb + j] = Cb[lb][j];
            K256[(4 * la + 3) * 16 + 4 * lb + 3] = Db[lb];
        }
    }
}

/* Debug/test entry: backflow 9x9 velocity tangent of one outlet triangle. */
void synth_backflow_tangent(const synth_params *p, const double *X9, const double *vel9, double *K81) {
    coefs cf; gen_alpha(p, &cf);
    double X[3][3], vel[3][3];
    for (int a = 0; a < 3; ++a)
        for (int r = 0; r < 3; ++r) { X[a][r] = X9[3 * a + r]; vel[a][r] = vel9[3 * a + r]; }
    for (int la = 0; la < 3; ++la) {
        double Ab[3][3][3];
        tri_backflow_rows(&cf, X, vel, la, Ab);
        for (int lb = 0; lb < 3; ++lb)
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) K81[(3 * la + i) * 9 + 3 * lb + j] = Ab[lb][i][j];
    }
}

static inline int find_col(const int32_t *col, int32_t beg, int32_t end, int32_t c) {
    for (int32_t e = beg; e < end; ++e)
        if (col[e] == c) return e;
    return -1;
}

/* Outlet piece of a top-face triangle with centroid (x, y in [0,1]) for
 * n_out pieces: 1 whole face, 2 halves in x, 3 thirds in x, 4 quadrants;
 * more than 4 (many-outlet stress cases): n_out patches of consecutive
 * triangles, triangle t of T (loop order: squares row by row, two
 * triangles each) in patch floor(t n_out / T), every patch non-empty when
 * n_out <= T. */
static inline int outlet_piece(int n_out, double x, double y, long t, long T) {
    if (n_out <= 1) return 0;
    if (n_out == 2) return x >= 0.5;
    if (n_out == 3) { int k = (int)(3.0 * x); return k > 2 ? 2 : k; }
    if (n_out == 4) return (x >= 0.5) + 2 * (y >= 0.5);
    return (int)((t * (long)n_out) / T);
}

/* Assemble the tangent on the shared pattern (rowptr/col from synth_pattern).
 * Aval 9 nnz, Bval 3 nnz, Cval 3 nnz, Dval nnz; avec = n_out dense 3N vectors
 * (outlet k at avec + 3N k).  Row-wise (one node per iteration), race-free and
 * independent of the thread count. */
int synth_assemble(const synth_params *p, const double *vel, const int32_t *rowptr, const int32_t *col,
                   double *Aval, double *Bval, double *Cval, double *Dval, double *avec) {
    coefs cf; gen_alpha(p, &cf);
    long N = synth_num_nodes(p);
    double hx = p->Lx / p->nx, hy = p->Ly / p->ny, hz = p->Lz / p->nz;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(| : bad)
    for (long A = 0; A < N; ++A) {
        int i = (int)(A % (p->nx + 1));
        int j = (int)((A / (p->nx + 1)) % (p->ny + 1));
        int k = (int)(A / ((long)(p->nx + 1) * (p->ny + 1)));
        int32_t beg = rowptr[A], end = rowptr[A + 1];
        for (int32_t e = beg; e < end; ++e) {
            for (int t = 0; t < 9; ++t) Aval[9 * (long)e + t] = 0.0;
            for (int t = 0; t < 3; ++t) { Bval[3 * (long)e + t] = 0.0; Cval[3 * (long)e + t] = 0.0; }
            Dval[e] = 0.0;
        }
        for (int hk = k - 1; hk <= k; ++hk)
            for (int hj = j - 1; hj <= j; ++hj)
                for (int hi = i - 1; hi <= i; ++hi) {
                    if (hi < 0 || hj < 0 || hk < 0 || hi >= p->nx || hj >= p->ny || hk >= p->nz) continue;
                    int cA = (i - hi) + 2 * (j - hj) + 4 * (k - hk);
                    for (int t = 0; t < 6; ++t) {
                        int c[4];
                        kuhn_tet(t, c);
                        int la = -1;
                        for (int v = 0; v < 4; ++v)
                            if (c[v] == cA) la = v;
                        if (la < 0) continue;
                        double X[4][3], vv[4][3];
                        long gid[4];
                        for (int v = 0; v < 4; ++v) {
                            int bi = hi + (c[v] & 1), bj = hj + ((c[v] >> 1) & 1), bk = hk + ((c[v] >> 2) & 1);
                            X[v][0] = bi * hx; X[v][1] = bj * hy; X[v][2] = bk * hz;
                            gid[v] = nid(p, bi, bj, bk);
                            for (int r = 0; r < 3; ++r) vv[v][r] = vel[3 * gid[v] + r];
                        }
                        double Ab[4][3][3], Bb[4][3], Cb[4][3], Db[4];
                        tet_rows(&cf, X, vv, la, Ab, Bb, Cb, Db);
                        for (int lb = 0; lb < 4; ++lb) {
                            int e = find_col(col, beg, end, (int32_t)gid[lb]);
                            if (e < 0) { bad = 1; continue; }
                            for (int r = 0; r < 3; ++r)
                                for (int s = 0; s < 3; ++s) Aval[9 * (long)e + 3 * r + s] += Ab[lb][r][s];
                            for (int r = 0; r < 3; ++r) {
                                Bval[3 * (long)e + r] += Bb[lb][r];
                                Cval[3 * (long)e + r] += Cb[lb][r];
                            }
                            Dval[e] += Db[lb];
                        }
                    }
                }
        /* backflow on the outlet face z = Lz: triangles (c4,c5,c7), (c4,c6,c7) of each top square */
        if (k == p->nz) {
            for (int hj = j - 1; hj <= j; ++hj)
                for (int hi = i - 1; hi <= i; ++hi) {
                    if (hi < 0 || hj < 0 || hi >= p->nx || hj >= p->ny) continue;
                    static const int tri[2][3] = {{0, 1, 3}, {0, 2, 3}}; /* corner codes on the face: bx + 2 by */
                    int cA = (i - hi) + 2 * (j - hj);
                    for (int t = 0; t < 2; ++t) {
                        int la = -1;
                        for (int v = 0; v < 3; ++v)
                            if (tri[t][v] == cA) la = v;
                        if (la < 0) continue;
                        double X[3][3], vv[3][3];
                        long gid[3];
                        for (int v = 0; v < 3; ++v) {
                            int bi = hi + (tri[t][v] & 1), bj = hj + ((tri[t][v] >> 1) & 1);
                            X[v][0] = bi * hx; X[v][1] = bj * hy; X[v][2] = p->Lz;
                            gid[v] = nid(p, bi, bj, p->nz);
                            for (int r = 0; r < 3; ++r) vv[v][r] = vel[3 * gid[v] + r];
                        }
                        double Ab[3][3][3];
                        tri_backflow_rows(&cf, X, vv, la, Ab);
                        for (int lb = 0; lb < 3; ++lb) {
                            int e = find_col(col, beg, end, (int32_t)gid[lb]);
                            if (e < 0) { bad = 1; continue; }
                            for (int r = 0; r < 3; ++r)
                                for (int s = 0; s < 3; ++s) Aval[9 * (long)e + 3 * r + s] += Ab[lb][r][s];
                        }
                    }
                }
        }
        /* Dirichlet treatment on this row and on Dirichlet columns */
        int dirA = is_dirichlet(p, i, j, k);
        for (int32_t e = beg; e < end; ++e) {
            long B = col[e];
            int bi = (int)(B % (p->nx + 1));
            int bj = (int)((B / (p->nx + 1)) % (p->ny + 1));
            int bk = (int)(B / ((long)(p->nx + 1) * (p->ny + 1)));
            int dirB = is_dirichlet(p, bi, bj, bk);
            for (int r = 0; r < 3; ++r)
                for (int s = 0; s < 3; ++s) {
                    int keep = (B == A && r == s) || (!dirA && !dirB);
                    if (!keep) Aval[9 * (long)e + 3 * r + s] = 0.0;
                }
            if (dirA)
                for (int r = 0; r < 3; ++r) Bval[3 * (long)e + r] = 0.0;
            if (dirB)
                for (int r = 0; r < 3; ++r) Cval[3 * (long)e + r] = 0.0;
        }
    }
    /* outlet vectors a^k_{A,z} = int_{Gamma_k} N_A dGamma (n = +e_z), zero at Dirichlet nodes */
    if (avec) {
        memset(avec, 0, sizeof(double) * 3 * (size_t)N * (size_t)(p->n_out > 0 ? p->n_out : 0));
        double area = 0.5 * hx * hy;
        for (int hj = 0; hj < p->ny; ++hj)
            for (int hi = 0; hi < p->nx; ++hi) {
                static const int tri[2][3] = {{0, 1, 3}, {0, 2, 3}};
                for (int t = 0; t < 2; ++t) {
                    double cx = 0.0, cy = 0.0;
                    for (int v = 0; v < 3; ++v) {
                        cx += (hi + (tri[t][v] & 1)) * hx;
                        cy += (hj + ((tri[t][v] >> 1) & 1)) * hy;
                    }
                    cx /= 3.0 * p->Lx; cy /= 3.0 * p->Ly;
                    int kk = outlet_piece(p->n_out, cx, cy, 2L * ((long)hj * p->nx + hi) + t, 2L * p->nx * p->ny);
                    for (int v = 0; v < 3; ++v) {
                        int bi = hi + (tri[t][v] & 1), bj = hj + ((tri[t][v] >> 1) & 1);
                        if (is_dirichlet(p, bi, bj, p->nz)) continue;
                        long g = nid(p, bi, bj, p->nz);
                        avec[3 * (size_t)N * kk + 3 * g + 2] += area / 3.0;
                    }
                }
            }
    }
    return bad ? -1 : 0;
}

/* Outlet vectors in sparse form, the same values as the dense avec of
 * synth_assemble (same triangles, same summation order): outlet k has
 * entries out_idx/out_val[out_ptr[k] .. out_ptr[k+1]-1], unknown indices
 * 3g + 2 (z component) ascending, Dirichlet nodes left out.  With out_idx ==
 * NULL only out_ptr is filled.  Returns the entry count, or -1 when
 * n_out exceeds the 2 nx ny outlet triangles. */
long synth_outlets(const synth_params *p, int32_t *out_ptr, int32_t *out_idx, double *out_val) {
    const int n_out = p->n_out > 0 ? p->n_out : 0;
    const long nf = (long)(p->nx + 1) * (p->ny + 1);
    if (n_out > 2L * p->nx * p->ny) return -1;
    if (n_out == 0) {   /* no outlets: nothing to assemble */
        if (out_ptr) out_ptr[0] = 0;
        return 0;
    }
    double *acc = (double *)calloc((size_t)n_out * (size_t)nf, sizeof(double));
    unsigned char *hit = (unsigned char *)calloc((size_t)n_out * (size_t)nf, 1);
    if ((n_out && !acc) || (n_out && !hit)) { free(acc); free(hit); return -1; }
    const double hx = p->Lx / p->nx, hy = p->Ly / p->ny;
    const double area = 0.5 * hx * hy;
    for (int hj = 0; hj < p->ny; ++hj)
        for (int hi = 0; hi < p->nx; ++hi) {
            static const int tri[2][3] = {{0, 1, 3}, {0, 2, 3}};
            for (int t = 0; t < 2; ++t) {
                double cx = 0.0, cy = 0.0;
                for (int v = 0; v < 3; ++v) {
                    cx += (hi + (tri[t][v] & 1)) * hx;
                    cy += (hj + ((tri[t][v] >> 1) & 1)) * hy;
                }
                cx /= 3.0 * p->Lx; cy /= 3.0 * p->Ly;
                int kk = outlet_piece(p->n_out, cx, cy, 2L * ((long)hj * p->nx + hi) + t, 2L * p->nx * p->ny);
                for (int v = 0; v < 3; ++v) {
                    int bi = hi + (tri[t][v] & 1), bj = hj + ((tri[t][v] >> 1) & 1);
                    if (is_dirichlet(p, bi, bj, p->nz)) continue;
                    long f = (long)bj * (p->nx + 1) + bi;
                    acc[(size_t)kk * nf + f] += area / 3.0;
                    hit[(size_t)kk * nf + f] = 1;
                }
            }
        }
    long cnt = 0;
    for (int k = 0; k < n_out; ++k) {
        if (out_ptr) out_ptr[k] = (int32_t)cnt;
        for (long f = 0; f < nf; ++f) {
            if (!hit[(size_t)k * nf + f] || acc[(size_t)k * nf + f] == 0.0) continue;
            if (out_idx) {
                int bi = (int)(f % (p->nx + 1)), bj = (int)(f / (p->nx + 1));
                out_idx[cnt] = (int32_t)(3 * nid(p, bi, bj, p->nz) + 2);
                out_val[cnt] = acc[(size_t)k * nf + f];
            }
            ++cnt;
        }
    }
    if (out_ptr) out_ptr[n_out] = (int32_t)cnt;
    free(acc);
    free(hit);
    return cnt;
}

/* Mesh arrays of the box (input data for a residual/tangent assembler):
 *   X        3N node coordinates (node ids as everywhere: x fastest);
 *   tets     4 node ids per tet, 6 nx ny nz tets (hex (hi, hj, hk) in x-fastest
 *            order, Kuhn tet t of that hex at 6 h + t, nodes in kuhn_tet order);
 *   tris     3 node ids per outlet triangle on z = Lz, 2 nx ny triangles
 *            (square (hi, hj) row by row, two triangles each), ordered so that
 *            (x1 - x0) x (x2 - x0) points out of the box (+e_z);
 *   tri_out  the outlet piece of each triangle (the partition of synth_outlets);
 *   dir      1 for each node whose velocity is prescribed (walls, inlet).
 * Any pointer may be NULL. */
void synth_mesh(const synth_params *p, double *X, int32_t *tets, int32_t *tris, int32_t *tri_out, uint8_t *dir) {
    const double hx = p->Lx / p->nx, hy = p->Ly / p->ny, hz = p->Lz / p->nz;
    for (int k = 0; k <= p->nz; ++k)
        for (int j = 0; j <= p->ny; ++j)
            for (int i = 0; i <= p->nx; ++i) {
                long a = nid(p, i, j, k);
                if (X) { X[3 * a] = i * hx; X[3 * a + 1] = j * hy; X[3 * a + 2] = k * hz; }
                if (dir) dir[a] = (uint8_t)is_dirichlet(p, i, j, k);
            }
    if (tets) {
        long e = 0;
        for (int hk = 0; hk < p->nz; ++hk)
            for (int hj = 0; hj < p->ny; ++hj)
                for (int hi = 0; hi < p->nx; ++hi)
                    for (int t = 0; t < 6; ++t, ++e) {
                        int c[4];
                        kuhn_tet(t, c);
                        for (int v = 0; v < 4; ++v)
                            tets[4 * e + v] = (int32_t)nid(p, hi + (c[v] & 1), hj + ((c[v] >> 1) & 1), hk + ((c[v] >> 2) & 1));
                    }
    }
    /* corner codes bx + 2 by on the top face; both triangles counter-clockwise seen from +z */
    static const int tri[2][3] = {{0, 1, 3}, {0, 3, 2}};
    for (int hj = 0; hj < p->ny; ++hj)
        for (int hi = 0; hi < p->nx; ++hi)
            for (int t = 0; t < 2; ++t) {
                long f = 2L * ((long)hj * p->nx + hi) + t;
                double cx = 0.0, cy = 0.0;
                for (int v = 0; v < 3; ++v) {
                    int bi = hi + (tri[t][v] & 1), bj = hj + ((tri[t][v] >> 1) & 1);
                    if (tris) tris[3 * f + v] = (int32_t)nid(p, bi, bj, p->nz);
                    cx += bi * hx; cy += bj * hy;
                }
                cx /= 3.0 * p->Lx; cy /= 3.0 * p->Ly;
                if (tri_out) tri_out[f] = p->n_out > 0 ? outlet_piece(p->n_out, cx, cy, f, 2L * p->nx * p->ny) : -1;
            }
}

/* Right-hand side: uniform [-1, 1] on all 4N unknowns, ordered [x_v (3N, node
 * interleaved); x_p (N)], drawn from a stream seeded with seed ^ 0xB0B. */
void synth_rhs(const synth_params *p, double *b) {
    uint64_t s = p->seed ^ 0xB0Bull;
    long n = 4 * synth_num_nodes(p);
    for (long i = 0; i < n; ++i) b[i] = 2.0 * sm64_u01(&s) - 1.0;
}

/* Stream of uniforms for the caller (outlet resistances, batch parameters). */
void synth_uniforms(uint64_t seed, long n, double *out) {
    uint64_t s = seed;
    for (long i = 0; i < n; ++i) out[i] = sm64_u01(&s);
}
