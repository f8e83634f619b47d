/*
 * vms_oracle.c -- TEST INFRASTRUCTURE (oracle), not the product path: only
 * tests/, the smoke check and the benchmark's CPU baseline may call it.
 *
 * Plain FP64 CPU restatement of the residual of the P1-P1 residual-based
 * variational multiscale (VMS) discretisation with generalized-alpha time
 * stepping, and of its consistent tangent:
 *
 *   R_m = R_m^vol + R_m^bc + R_m^bf   (Sec. 2.3, B_m^vol, B_m^bc, B_m^bf)
 *   R_p                                (Sec. 2.3, B_p)
 *
 * evaluated at (vdot_{n+alpha_m}, v_{n+alpha_f}, p_{n+alpha_f}) (Sec. 2.4:
 * the pressure is taken at n+alpha_f), with the fine scales
 * v' = -tau_M (rho vdot + rho v.grad v + grad p - mu lap v - rho b) and
 * p' = -tau_C div v, tau_M, tau_C and the metric G as defined in Sec. 2.3
 * (C_I = 36, C_T = 4, M = 2^(1/3)/2 [[2,1,1],[1,2,1],[1,1,2]]).  For P1
 * elements lap v vanishes inside each element; the body force b is zero.
 *
 * The tangent (Sec. 2.5, definitions of A = F + K, B, C, D) is the derivative
 * of that residual with respect to the unknowns (vdot_{n+1}, pdot_{n+1}):
 * d/dvdot_{n+1} = alpha_m d/dvdot_{n+alpha_m} + alpha_f gamma dt d/dv_{n+alpha_f}
 * and d/dpdot_{n+1} = alpha_f gamma dt d/dp_{n+alpha_f}.  It is taken exactly,
 * by forward-mode dual numbers carrying the 16 partials of one element (the
 * 4 unknowns of each of its 4 nodes), with tau_M and tau_C frozen at the
 * state (reading: the paper does not say whether the stabilisation
 * parameters are differentiated; freezing them is the usual choice).  The
 * resistance part K = alpha_f gamma dt sum_k m^k a^k a^kT is not assembled:
 * it stays the matrix-free rank-one term of the solvers.
 *
 * Dirichlet nodes (all three velocity components prescribed): their momentum
 * residual rows are zero; in the tangent their velocity rows and columns keep
 * only the diagonal entry, their B rows and C columns are zero.
 *
 * Unknown layout: velocity 3N node-interleaved, then pressure N (as the
 * solvers' x = [x_v; x_p]).  Tangent on the shared block pattern
 * (rowptr, col): A 9 values per entry (row-major 3x3), B 3 (column vector),
 * C 3 (row vector), D 1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ND 16   /* partials: unknown (node lb, dof d) -> 4 lb + d, d = 3 pressure */

typedef struct {
    double v;
    double d[ND];
} dual;

typedef struct {
    double rho, mu, dt, rho_inf, beta, CI, CT;
} or_vms_phys;

static dual dcon(double v) {
    dual r;
    r.v = v;
    memset(r.d, 0, sizeof r.d);
    return r;
}
static dual dadd(dual a, dual b) {
    a.v += b.v;
    for (int i = 0; i < ND; ++i) a.d[i] += b.d[i];
    return a;
}
static dual dsub(dual a, dual b) {
    a.v -= b.v;
    for (int i = 0; i < ND; ++i) a.d[i] -= b.d[i];
    return a;
}
static dual dmul(dual a, dual b) {
    dual r;
    r.v = a.v * b.v;
    for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
}
static dual dscl(dual a, double s) {
    a.v *= s;
    for (int i = 0; i < ND; ++i) a.d[i] *= s;
    return a;
}

/* generalized-alpha parameters from rho_inf (Sec. 2.4.1) */
static void gen_alpha(double rho_inf, double *am, double *af, double *gm) {
    *am = 0.5 * (3.0 - rho_inf) / (1.0 + rho_inf);
    *af = 1.0 / (1.0 + rho_inf);
    *gm = 1.0 / (1.0 + rho_inf);
}

/* Gradients of the four P1 shape functions (rows) and the tet volume.
 * With the parent coordinates xi_k = N_k (k = 1..3), the Jacobian
 * J_rk = dx_r/dxi_k = x_k - x_0; dxi/dx = J^{-1} from the adjugate. */
static double tet_gradients(const double X[4][3], double dN[4][3]) {
    double J[3][3], adj[3][3];
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) J[r][k] = X[k + 1][r] - X[0][r];
    adj[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    adj[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    adj[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    adj[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    adj[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    adj[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    adj[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    adj[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    adj[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    const double det = J[0][0] * adj[0][0] + J[0][1] * adj[1][0] + J[0][2] * adj[2][0];
    /* (J^{-1})_kr = adj_kr / det = dxi_k / dx_r */
    for (int r = 0; r < 3; ++r) {
        double s = 0.0;
        for (int k = 0; k < 3; ++k) {
            dN[k + 1][r] = adj[k][r] / det;
            s += dN[k + 1][r];
        }
        dN[0][r] = -s;
    }
    return fabs(det) / 6.0;
}

/* G_ij = sum_kl dxi_k/dx_i M_kl dxi_l/dx_j (Sec. 2.3) */
static void metric(const double dN[4][3], double G[3][3]) {
    const double c = cbrt(2.0) / 2.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double g = 0.0;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) g += dN[k + 1][i] * (c * (k == l ? 2.0 : 1.0)) * dN[l + 1][j];
            G[i][j] = g;
        }
}

static int slot_of(const int32_t *rowptr, const int32_t *col, int A, int B) {
    for (int32_t e = rowptr[A]; e < rowptr[A + 1]; ++e)
        if (col[e] == B) return e;
    return -1;
}

/* Element residual rows (Rm[la][i], Rp[la]) as duals over the element's 16
 * unknowns.  vd, v, p: nodal states; vt: the velocity tau is evaluated at. */
static void tet_residual(const or_vms_phys *ph, double am, double afgdt, const double X[4][3], const double vd[4][3],
                         const double v[4][3], const double p[4], const double vt[4][3], dual Rm[4][3], dual Rp[4]) {
    double dN[4][3], G[3][3];
    const double vol = tet_gradients(X, dN);
    metric(dN, G);
    double GG = 0.0, trG = 0.0;
    for (int i = 0; i < 3; ++i) {
        trG += G[i][i];
        for (int j = 0; j < 3; ++j) GG += G[i][j] * G[i][j];
    }
    const double rho = ph->rho, mu = ph->mu;
    /* seeded nodal unknowns */
    dual VD[4][3], V[4][3], P[4];
    for (int b = 0; b < 4; ++b) {
        for (int i = 0; i < 3; ++i) {
            VD[b][i] = dcon(vd[b][i]);
            VD[b][i].d[4 * b + i] = am;
            V[b][i] = dcon(v[b][i]);
            V[b][i].d[4 * b + i] = afgdt;
        }
        P[b] = dcon(p[b]);
        P[b].d[4 * b + 3] = afgdt;
    }
    /* element-constant gradients: Gv_ij = d v_i / d x_j, grad p, div v */
    dual Gv[3][3], gp[3], div = dcon(0.0);
    for (int i = 0; i < 3; ++i) {
        gp[i] = dcon(0.0);
        for (int b = 0; b < 4; ++b) gp[i] = dadd(gp[i], dscl(P[b], dN[b][i]));
        for (int j = 0; j < 3; ++j) {
            Gv[i][j] = dcon(0.0);
            for (int b = 0; b < 4; ++b) Gv[i][j] = dadd(Gv[i][j], dscl(V[b][i], dN[b][j]));
        }
    }
    for (int i = 0; i < 3; ++i) div = dadd(div, Gv[i][i]);
    for (int a = 0; a < 4; ++a) {
        Rp[a] = dcon(0.0);
        for (int i = 0; i < 3; ++i) Rm[a][i] = dcon(0.0);
    }
    /* 4-point rule, degree 2: barycentric (a, b, b, b) and permutations */
    const double qa = (5.0 + 3.0 * sqrt(5.0)) / 20.0, qb = (5.0 - sqrt(5.0)) / 20.0;
    const double w = vol / 4.0;
    for (int q = 0; q < 4; ++q) {
        double N[4];
        for (int b = 0; b < 4; ++b) N[b] = (b == q) ? qa : qb;
        dual u[3], ud[3], pq = dcon(0.0);
        double ut[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < 3; ++i) {
            u[i] = dcon(0.0);
            ud[i] = dcon(0.0);
            for (int b = 0; b < 4; ++b) {
                u[i] = dadd(u[i], dscl(V[b][i], N[b]));
                ud[i] = dadd(ud[i], dscl(VD[b][i], N[b]));
                ut[i] += N[b] * vt[b][i];
            }
        }
        for (int b = 0; b < 4; ++b) pq = dadd(pq, dscl(P[b], N[b]));
        /* tau_M, tau_C at the frozen velocity */
        double uGu = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) uGu += ut[i] * G[i][j] * ut[j];
        const double tauM = 1.0 / (rho * sqrt(ph->CT / (ph->dt * ph->dt) + uGu + ph->CI * (mu / rho) * (mu / rho) * GG));
        const double tauC = 1.0 / (tauM * trG);
        /* (v . grad) v, the strong momentum residual and the fine scales */
        dual conv[3], vp[3];
        for (int i = 0; i < 3; ++i) {
            conv[i] = dcon(0.0);
            for (int j = 0; j < 3; ++j) conv[i] = dadd(conv[i], dmul(Gv[i][j], u[j]));
            dual rM = dadd(dadd(dscl(ud[i], rho), dscl(conv[i], rho)), gp[i]);
            vp[i] = dscl(rM, -tauM);
        }
        const dual pp = dscl(div, -tauC);
        for (int a = 0; a < 4; ++a) {
            dual u_dNa = dcon(0.0), vp_dNa = dcon(0.0);
            for (int j = 0; j < 3; ++j) {
                u_dNa = dadd(u_dNa, dscl(u[j], dN[a][j]));
                vp_dNa = dadd(vp_dNa, dscl(vp[j], dN[a][j]));
            }
            for (int i = 0; i < 3; ++i) {
                /* w . rho (dv/dt + v . grad v) */
                dual t = dscl(dadd(ud[i], conv[i]), rho * N[a]);
                /* - div w p */
                t = dsub(t, dscl(pq, dN[a][i]));
                /* 2 mu eps(w) : eps(v) = mu sum_j dN_a,j (dv_i/dx_j + dv_j/dx_i) */
                for (int j = 0; j < 3; ++j) t = dadd(t, dscl(dadd(Gv[i][j], Gv[j][i]), mu * dN[a][j]));
                /* - grad w : (rho v' (x) v) */
                t = dsub(t, dscl(dmul(vp[i], u_dNa), rho));
                /* + grad v : (rho w (x) v') */
                dual gvv = dcon(0.0);
                for (int j = 0; j < 3; ++j) gvv = dadd(gvv, dmul(Gv[i][j], vp[j]));
                t = dadd(t, dscl(gvv, rho * N[a]));
                /* - grad w : (rho v' (x) v') */
                t = dsub(t, dscl(dmul(vp[i], vp_dNa), rho));
                /* - div w p' */
                t = dsub(t, dscl(pp, dN[a][i]));
                Rm[a][i] = dadd(Rm[a][i], dscl(t, w));
            }
            /* q div v - grad q . v' */
            Rp[a] = dadd(Rp[a], dscl(dsub(dscl(div, N[a]), vp_dNa), w));
        }
    }
}

/* Backflow rows of one outlet triangle (B_m^bf, Sec. 2.3): -rho beta
 * (v.n)_- w.v, 3-point rule at the edge midpoints' dual points
 * (barycentric (2/3, 1/6, 1/6) and permutations), n the outward unit normal
 * (x1 - x0) x (x2 - x0) / |.|.  Partials at 4 lb + i as in tet_residual. */
static void tri_backflow(const or_vms_phys *ph, double afgdt, const double X[3][3], const double v[3][3],
                         dual Rm[3][3]) {
    double e1[3], e2[3], n[3];
    for (int r = 0; r < 3; ++r) { e1[r] = X[1][r] - X[0][r]; e2[r] = X[2][r] - X[0][r]; }
    n[0] = e1[1] * e2[2] - e1[2] * e2[1];
    n[1] = e1[2] * e2[0] - e1[0] * e2[2];
    n[2] = e1[0] * e2[1] - e1[1] * e2[0];
    const double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    for (int r = 0; r < 3; ++r) n[r] /= len;
    const double w = 0.5 * len / 3.0;
    dual V[3][3];
    for (int b = 0; b < 3; ++b)
        for (int i = 0; i < 3; ++i) {
            V[b][i] = dcon(v[b][i]);
            V[b][i].d[4 * b + i] = afgdt;
        }
    for (int a = 0; a < 3; ++a)
        for (int i = 0; i < 3; ++i) Rm[a][i] = dcon(0.0);
    for (int q = 0; q < 3; ++q) {
        double N[3];
        for (int b = 0; b < 3; ++b) N[b] = (b == q) ? 2.0 / 3.0 : 1.0 / 6.0;
        dual u[3], un = dcon(0.0);
        for (int i = 0; i < 3; ++i) {
            u[i] = dcon(0.0);
            for (int b = 0; b < 3; ++b) u[i] = dadd(u[i], dscl(V[b][i], N[b]));
            un = dadd(un, dscl(u[i], n[i]));
        }
        if (!(un.v < 0.0)) continue;   /* (v.n)_- = v.n where negative, else 0 */
        for (int a = 0; a < 3; ++a)
            for (int i = 0; i < 3; ++i)
                Rm[a][i] = dadd(Rm[a][i], dscl(dmul(un, u[i]), -ph->rho * ph->beta * N[a] * w));
    }
}

/* Residual R (4N, or NULL) and tangent values (or NULL) at the state
 * (vd = vdot_{n+alpha_m}, v = v_{n+alpha_f}, p = p_{n+alpha_f}), outlet
 * pressures P_k = P^k_{n+alpha_f} entering R_m^bc = sum_k P_k a^k (a^k the
 * sparse outlet vectors optr/oidx/oval over velocity dofs), tau evaluated at
 * vtau (NULL: v).  tris: the Neumann boundary triangles (backflow).
 * Returns 0, or -1 when an element couples two nodes absent from the pattern. */
int or_vms_assemble(int N, const double *Xn, int E, const int32_t *tets, int T, const int32_t *tris,
                    const uint8_t *dirn, const or_vms_phys *ph, const double *vd, const double *v, const double *p,
                    const double *vtau, int n_out, const int32_t *optr, const int32_t *oidx, const double *oval,
                    const double *Pk, const int32_t *rowptr, const int32_t *col, double *R, double *Aval,
                    double *Bval, double *Cval, double *Dval) {
    double am, af, gm;
    gen_alpha(ph->rho_inf, &am, &af, &gm);
    const double afgdt = af * gm * ph->dt;
    const int tang = Aval && Bval && Cval && Dval;
    const int64_t nnz = rowptr[N];
    if (!vtau) vtau = v;
    if (R) memset(R, 0, sizeof(double) * 4 * (size_t)N);
    if (tang) {
        memset(Aval, 0, sizeof(double) * 9 * (size_t)nnz);
        memset(Bval, 0, sizeof(double) * 3 * (size_t)nnz);
        memset(Cval, 0, sizeof(double) * 3 * (size_t)nnz);
        memset(Dval, 0, sizeof(double) * (size_t)nnz);
    }
    int bad = 0;
    for (int e = 0; e < E; ++e) {
        double X[4][3], VD[4][3], V[4][3], P[4], VT[4][3];
        const int32_t *nd = tets + 4 * (size_t)e;
        for (int b = 0; b < 4; ++b) {
            for (int r = 0; r < 3; ++r) {
                X[b][r] = Xn[3 * (size_t)nd[b] + r];
                VD[b][r] = vd[3 * (size_t)nd[b] + r];
                V[b][r] = v[3 * (size_t)nd[b] + r];
                VT[b][r] = vtau[3 * (size_t)nd[b] + r];
            }
            P[b] = p[nd[b]];
        }
        dual Rm[4][3], Rp[4];
        tet_residual(ph, am, afgdt, X, VD, V, P, VT, Rm, Rp);
        for (int a = 0; a < 4; ++a) {
            const int A = nd[a];
            if (R) {
                for (int i = 0; i < 3; ++i) R[3 * (size_t)A + i] += Rm[a][i].v;
                R[3 * (size_t)N + A] += Rp[a].v;
            }
            if (!tang) continue;
            for (int b = 0; b < 4; ++b) {
                const int s = slot_of(rowptr, col, A, nd[b]);
                if (s < 0) { bad = 1; continue; }
                for (int i = 0; i < 3; ++i) {
                    for (int j = 0; j < 3; ++j) Aval[9 * (size_t)s + 3 * i + j] += Rm[a][i].d[4 * b + j];
                    Bval[3 * (size_t)s + i] += Rm[a][i].d[4 * b + 3];
                    Cval[3 * (size_t)s + i] += Rp[a].d[4 * b + i];
                }
                Dval[s] += Rp[a].d[4 * b + 3];
            }
        }
    }
    for (int t = 0; t < T; ++t) {
        double X[3][3], V[3][3];
        const int32_t *nd = tris + 3 * (size_t)t;
        for (int b = 0; b < 3; ++b)
            for (int r = 0; r < 3; ++r) {
                X[b][r] = Xn[3 * (size_t)nd[b] + r];
                V[b][r] = v[3 * (size_t)nd[b] + r];
            }
        dual Rm[3][3];
        tri_backflow(ph, afgdt, X, V, Rm);
        for (int a = 0; a < 3; ++a) {
            const int A = nd[a];
            if (R)
                for (int i = 0; i < 3; ++i) R[3 * (size_t)A + i] += Rm[a][i].v;
            if (!tang) continue;
            for (int b = 0; b < 3; ++b) {
                const int s = slot_of(rowptr, col, A, nd[b]);
                if (s < 0) { bad = 1; continue; }
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) Aval[9 * (size_t)s + 3 * i + j] += Rm[a][i].d[4 * b + j];
            }
        }
    }
    /* outlet traction: -int w.h with h = -P_k n on outlet k gives sum_k P_k a^k */
    if (R && Pk)
        for (int k = 0; k < n_out; ++k)
            for (int32_t q = optr[k]; q < optr[k + 1]; ++q) R[oidx[q]] += Pk[k] * oval[q];
    /* Dirichlet nodes */
    for (int A = 0; A < N; ++A) {
        if (R && dirn[A])
            for (int i = 0; i < 3; ++i) R[3 * (size_t)A + i] = 0.0;
        if (!tang) continue;
        for (int32_t s = rowptr[A]; s < rowptr[A + 1]; ++s) {
            const int B = col[s];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    const int keep = (A == B && i == j) || (!dirn[A] && !dirn[B]);
                    if (!keep) Aval[9 * (size_t)s + 3 * i + j] = 0.0;
                }
            if (dirn[A])
                for (int i = 0; i < 3; ++i) Bval[3 * (size_t)s + i] = 0.0;
            if (dirn[B])
                for (int i = 0; i < 3; ++i) Cval[3 * (size_t)s + i] = 0.0;
        }
    }
    return bad ? -1 : 0;
}
