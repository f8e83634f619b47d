// vms.cu -- on-device assembly of the residual and of the consistent tangent
// of the P1-P1 residual-based VMS / generalized-alpha discretisation.
//
// Residual (Sec. 2.3, B_m^vol + B_m^bc + B_m^bf and B_p, evaluated at
// vdot_{n+alpha_m}, v_{n+alpha_f}, p_{n+alpha_f} as Sec. 2.4 prescribes):
// per quadrature point of a tet, with u = v_h, the fine scales
// v' = -tau_M (rho udot + rho (u.grad) u + grad p) (P1: the viscous second
// derivatives vanish inside an element; no body force) and p' = -tau_C div u,
// the momentum row of node a, component i, gains
//   rho N_a (udot_i + (u.grad u)_i) - dN_a/dx_i p + mu dN_a/dx_j (du_i/dx_j + du_j/dx_i)
//   - rho v'_i (u.grad N_a) + rho N_a (v'.grad) u_i - rho v'_i (v'.grad N_a) - dN_a/dx_i p'
// and the continuity row N_a div u - grad N_a . v'.  tau_M, tau_C follow
// Sec. 2.3 (C_T, C_I, the metric G with the simplex matrix M), evaluated at a
// given velocity (the state itself, or a frozen one).  The outlet traction
// adds sum_k P_k a^k; backflow (B_m^bf) adds -rho beta (u.n)_- N_a u_i on the
// outlet triangles.
//
// Tangent (Sec. 2.5, F + the blocks B, C, D; K stays the solvers' matrix-free
// rank-one term): the derivative of the residual with respect to
// (vdot_{n+1}, pdot_{n+1}), i.e. alpha_m d/dvdot_{n+alpha_m} + alpha_f gamma
// dt d/d(v, p)_{n+alpha_f}, with tau_M and tau_C held fixed.  It is taken
// exactly by forward-mode dual numbers with four partials: one thread per
// (tet, column node b) seeds the four unknowns of b and evaluates the tet's
// four rows, which gives the four 4x4 blocks of column b.
//
// Determinism: every tet (triangle) writes its own scratch slots; gather
// kernels then sum, per residual row and per pattern slot, the slots of the
// incident elements in ascending element order.  No atomics.
#include "nbp_common.cuh"
#include "vms.cuh"

namespace nbp {

// ---------------------------------------------------------------- dual numbers
template <typename T> struct D4 {
    T v, d[4];
};
template <typename T> __device__ __forceinline__ D4<T> operator+(D4<T> a, const D4<T> &b) {
    a.v += b.v;
#pragma unroll
    for (int q = 0; q < 4; ++q) a.d[q] += b.d[q];
    return a;
}
template <typename T> __device__ __forceinline__ D4<T> operator-(D4<T> a, const D4<T> &b) {
    a.v -= b.v;
#pragma unroll
    for (int q = 0; q < 4; ++q) a.d[q] -= b.d[q];
    return a;
}
template <typename T> __device__ __forceinline__ D4<T> operator*(const D4<T> &a, const D4<T> &b) {
    D4<T> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int q = 0; q < 4; ++q) r.d[q] = a.d[q] * b.v + a.v * b.d[q];
    return r;
}
template <typename T> __device__ __forceinline__ D4<T> operator*(D4<T> a, T s) {
    a.v *= s;
#pragma unroll
    for (int q = 0; q < 4; ++q) a.d[q] *= s;
    return a;
}

// uniform access for plain and dual values
template <typename V> struct Num;
template <> struct Num<double> {
    using T = double;
    __device__ static double cst(double c) { return c; }
    __device__ static double val(double x) { return x; }
};
template <typename T_> struct Num<D4<T_>> {
    using T = T_;
    __device__ static D4<T_> cst(T_ c) {
        D4<T_> r;
        r.v = c;
#pragma unroll
        for (int q = 0; q < 4; ++q) r.d[q] = T_(0);
        return r;
    }
    __device__ static T_ val(const D4<T_> &x) { return x.v; }
};

// ---------------------------------------------------------------- geometry
// Barycentric gradients by cross products: grad l_1 = (e2 x e3) / det, etc.,
// e_k = x_k - x_0, det = e1 . (e2 x e3), grad l_0 = -(sum of the others).
// G = m0 sum_{a=0..3} grad l_a (x) grad l_a: with xi_k = l_k (k = 1..3) and
// M = m0 (1 + delta_kl), sum_kl dxi_k M_kl dxi_l expands to exactly this.
template <typename T> struct Geo {
    T dN[4][3];
    T vol, G[3][3], GG, trG;
};
template <typename T> __device__ __forceinline__ void cross3(const T a[3], const T b[3], T c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
template <typename T> __device__ void tet_geo(const double *X, const int *nd, Geo<T> &g) {
    T x0[3], e[3][3];
    for (int r = 0; r < 3; ++r) x0[r] = (T)X[3LL * nd[0] + r];
    for (int k = 0; k < 3; ++k)
        for (int r = 0; r < 3; ++r) e[k][r] = (T)X[3LL * nd[k + 1] + r] - x0[r];
    T c23[3], c31[3], c12[3];
    cross3(e[1], e[2], c23);
    cross3(e[2], e[0], c31);
    cross3(e[0], e[1], c12);
    const T det = e[0][0] * c23[0] + e[0][1] * c23[1] + e[0][2] * c23[2];
    const T inv = T(1) / det;
    for (int r = 0; r < 3; ++r) {
        g.dN[1][r] = c23[r] * inv;
        g.dN[2][r] = c31[r] * inv;
        g.dN[3][r] = c12[r] * inv;
        g.dN[0][r] = -(g.dN[1][r] + g.dN[2][r] + g.dN[3][r]);
    }
    g.vol = fabs(det) / T(6);
    const T m0 = T(0.62996052494743658238);   // 2^(1/3) / 2
    g.GG = T(0);
    g.trG = T(0);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            T s = T(0);
            for (int a = 0; a < 4; ++a) s += g.dN[a][i] * g.dN[a][j];
            g.G[i][j] = m0 * s;
            g.GG += g.G[i][j] * g.G[i][j];
        }
    g.trG = g.G[0][0] + g.G[1][1] + g.G[2][2];
}

// ------------------------------------------------------------ element rows
// Rows of all four nodes of one tet: Rm[a][i] (momentum), Rp[a] (continuity).
// UD, U, P: nodal vdot, v, p (plain or seeded duals); UT: the velocity tau is
// evaluated at.
template <typename V>
__device__ void tet_rows(const VmsConst &k, const Geo<typename Num<V>::T> &g, const V UD[4][3], const V U[4][3],
                         const V P[4], const typename Num<V>::T UT[4][3], V Rm[4][3], V Rp[4]) {
    using T = typename Num<V>::T;
    using Nm = Num<V>;
    const T rho = (T)k.rho, mu = (T)k.mu;
    V Gv[3][3], gp[3];
    for (int i = 0; i < 3; ++i) {
        gp[i] = P[0] * g.dN[0][i] + P[1] * g.dN[1][i] + P[2] * g.dN[2][i] + P[3] * g.dN[3][i];
        for (int j = 0; j < 3; ++j)
            Gv[i][j] = U[0][i] * g.dN[0][j] + U[1][i] * g.dN[1][j] + U[2][i] * g.dN[2][j] + U[3][i] * g.dN[3][j];
    }
    const V dv = Gv[0][0] + Gv[1][1] + Gv[2][2];
    for (int a = 0; a < 4; ++a) {
        Rp[a] = Nm::cst(T(0));
        for (int i = 0; i < 3; ++i) Rm[a][i] = Nm::cst(T(0));
    }
    const T q_hi = T(0.58541019662496845446), q_lo = T(0.13819660112501051518);   // (5 + 3 sqrt5)/20, (5 - sqrt5)/20
    const T w = g.vol * T(0.25);
    const T visc2 = T(k.CI) * (mu / rho) * (mu / rho) * g.GG + T(k.CT / (k.dt * k.dt));
    for (int q = 0; q < 4; ++q) {
        T Nq[4];
        for (int b = 0; b < 4; ++b) Nq[b] = (b == q) ? q_hi : q_lo;
        V u[3], ud[3];
        T ut[3];
        for (int i = 0; i < 3; ++i) {
            u[i] = U[0][i] * Nq[0] + U[1][i] * Nq[1] + U[2][i] * Nq[2] + U[3][i] * Nq[3];
            ud[i] = UD[0][i] * Nq[0] + UD[1][i] * Nq[1] + UD[2][i] * Nq[2] + UD[3][i] * Nq[3];
            ut[i] = UT[0][i] * Nq[0] + UT[1][i] * Nq[1] + UT[2][i] * Nq[2] + UT[3][i] * Nq[3];
        }
        const V pq = P[0] * Nq[0] + P[1] * Nq[1] + P[2] * Nq[2] + P[3] * Nq[3];
        T uGu = T(0);
        for (int i = 0; i < 3; ++i) uGu += ut[i] * (g.G[i][0] * ut[0] + g.G[i][1] * ut[1] + g.G[i][2] * ut[2]);
        const T tauM = T(1) / (rho * sqrt(visc2 + uGu));
        const T tauC = T(1) / (tauM * g.trG);
        V cv[3], vp[3];
        for (int i = 0; i < 3; ++i) {
            cv[i] = Gv[i][0] * u[0] + Gv[i][1] * u[1] + Gv[i][2] * u[2];
            vp[i] = (ud[i] * rho + cv[i] * rho + gp[i]) * (-tauM);
        }
        const V pf = dv * (-tauC);
        V gvp[3];
        for (int i = 0; i < 3; ++i) gvp[i] = Gv[i][0] * vp[0] + Gv[i][1] * vp[1] + Gv[i][2] * vp[2];
        for (int a = 0; a < 4; ++a) {
            const T *d = g.dN[a];
            const V udN = u[0] * d[0] + u[1] * d[1] + u[2] * d[2];
            const V vdN = vp[0] * d[0] + vp[1] * d[1] + vp[2] * d[2];
            const V adv = (udN + vdN) * rho;   // rho (u + v') . grad N_a
            for (int i = 0; i < 3; ++i) {
                V t = (ud[i] + cv[i] + gvp[i]) * (rho * Nq[a]);
                t = t - (pq + pf) * d[i];
                t = t + ((Gv[i][0] + Gv[0][i]) * d[0] + (Gv[i][1] + Gv[1][i]) * d[1] + (Gv[i][2] + Gv[2][i]) * d[2]) * mu;
                t = t - vp[i] * adv;
                Rm[a][i] = Rm[a][i] + t * w;
            }
            Rp[a] = Rp[a] + (dv * Nq[a] - vdN) * w;
        }
    }
}

// Backflow rows of one outlet triangle: -rho beta (u.n)_- N_a u_i with the
// 3-point rule at barycentric (2/3, 1/6, 1/6) and its permutations.
template <typename V>
__device__ void tri_rows(const VmsConst &k, const double *X, const int *nd, const V U[3][3], V Rm[3][3]) {
    using T = typename Num<V>::T;
    using Nm = Num<V>;
    T e1[3], e2[3], n[3];
    for (int r = 0; r < 3; ++r) {
        e1[r] = (T)(X[3LL * nd[1] + r] - X[3LL * nd[0] + r]);
        e2[r] = (T)(X[3LL * nd[2] + r] - X[3LL * nd[0] + r]);
    }
    cross3(e1, e2, n);
    const T len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    for (int r = 0; r < 3; ++r) n[r] /= len;
    const T w = len / T(6);   // area / 3
    const T c = -(T)(k.rho * k.beta);
    for (int a = 0; a < 3; ++a)
        for (int i = 0; i < 3; ++i) Rm[a][i] = Nm::cst(T(0));
    for (int q = 0; q < 3; ++q) {
        T Nq[3];
        for (int b = 0; b < 3; ++b) Nq[b] = (b == q) ? T(2) / T(3) : T(1) / T(6);
        V u[3];
        for (int i = 0; i < 3; ++i) u[i] = U[0][i] * Nq[0] + U[1][i] * Nq[1] + U[2][i] * Nq[2];
        const V un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
        if (!(Nm::val(un) < T(0))) continue;
        for (int a = 0; a < 3; ++a)
            for (int i = 0; i < 3; ++i) Rm[a][i] = Rm[a][i] + (un * u[i]) * (c * Nq[a] * w);
    }
}

// ------------------------------------------------------------------ residual
__global__ void k_res_tet(int E, const double *X, const int *tets, const double *vd, const double *v, const double *p,
                          const double *vt, VmsConst k, double *Re) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    int nd[4];
    for (int a = 0; a < 4; ++a) nd[a] = tets[4LL * e + a];
    Geo<double> g;
    tet_geo<double>(X, nd, g);
    double UD[4][3], U[4][3], P[4], UT[4][3];
    for (int b = 0; b < 4; ++b) {
        for (int i = 0; i < 3; ++i) {
            UD[b][i] = vd[3LL * nd[b] + i];
            U[b][i] = v[3LL * nd[b] + i];
            UT[b][i] = vt[3LL * nd[b] + i];
        }
        P[b] = p[nd[b]];
    }
    double Rm[4][3], Rp[4];
    tet_rows<double>(k, g, UD, U, P, UT, Rm, Rp);
    for (int a = 0; a < 4; ++a) {
        double *o = Re + 16LL * e + 4 * a;
        o[0] = Rm[a][0];
        o[1] = Rm[a][1];
        o[2] = Rm[a][2];
        o[3] = Rp[a];
    }
}

__global__ void k_res_tri(int T, const double *X, const int *tris, const double *v, VmsConst k, double *Rf) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    int nd[3];
    for (int a = 0; a < 3; ++a) nd[a] = tris[3LL * t + a];
    double U[3][3], Rm[3][3];
    for (int b = 0; b < 3; ++b)
        for (int i = 0; i < 3; ++i) U[b][i] = v[3LL * nd[b] + i];
    tri_rows<double>(k, X, nd, U, Rm);
    for (int a = 0; a < 3; ++a)
        for (int i = 0; i < 3; ++i) Rf[9LL * t + 3 * a + i] = Rm[a][i];
}

// R rows of node A: its tets' rows (ascending e), its triangles' rows
// (ascending t), the outlet traction sum_k P_k a^k; Dirichlet momentum rows 0.
__global__ void k_res_gather(int N, const int *n2t_ptr, const int *n2t, const int *n2f_ptr, const int *n2f,
                             const double *Re, const double *Rf, const int *lr_rp, const int *lr_k, const int *lr_c,
                             const double *lr_v, const double *P, const uint8_t *dir, double *R) {
    const int A = blockIdx.x * blockDim.x + threadIdx.x;
    if (A >= N) return;
    double r0 = 0.0, r1 = 0.0, r2 = 0.0, r3 = 0.0;
    for (int q = n2t_ptr[A]; q < n2t_ptr[A + 1]; ++q) {
        const double *s = Re + 4LL * n2t[q];   // 16 e + 4 la
        r0 += s[0];
        r1 += s[1];
        r2 += s[2];
        r3 += s[3];
    }
    for (int q = n2f_ptr[A]; q < n2f_ptr[A + 1]; ++q) {
        const double *s = Rf + 3LL * n2f[q];   // 9 t + 3 la
        r0 += s[0];
        r1 += s[1];
        r2 += s[2];
    }
    if (P && lr_rp)
        for (int j = lr_rp[A]; j < lr_rp[A + 1]; ++j) {
            const double f = P[lr_k[j]] * lr_v[j];
            const int c = lr_c[j];
            if (c == 0) r0 += f;
            else if (c == 1) r1 += f;
            else r2 += f;
        }
    if (dir[A]) r0 = r1 = r2 = 0.0;
    R[3LL * A] = r0;
    R[3LL * A + 1] = r1;
    R[3LL * A + 2] = r2;
    R[3LL * N + A] = r3;
}

// ------------------------------------------------------------------- tangent
// Thread (e, b): seeds the unknowns of local node b -- vdot with alpha_m and
// v with alpha_f gamma dt (partials 0..2), p with alpha_f gamma dt (partial 3)
// -- and writes the blocks (a, b) of all four rows a.
template <typename T>
__global__ void k_tan_tet(int E, const double *X, const int *tets, const double *vd, const double *v, const double *p,
                          const double *vt, VmsConst k, T *Ke) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= 4LL * E) return;
    const int e = (int)(tid >> 2), b = (int)(tid & 3);
    int nd[4];
    for (int a = 0; a < 4; ++a) nd[a] = tets[4LL * e + a];
    Geo<T> g;
    tet_geo<T>(X, nd, g);
    D4<T> UD[4][3], U[4][3], P[4];
    T UT[4][3];
    for (int c = 0; c < 4; ++c) {
        for (int i = 0; i < 3; ++i) {
            UD[c][i] = Num<D4<T>>::cst((T)vd[3LL * nd[c] + i]);
            U[c][i] = Num<D4<T>>::cst((T)v[3LL * nd[c] + i]);
            UT[c][i] = (T)vt[3LL * nd[c] + i];
        }
        P[c] = Num<D4<T>>::cst((T)p[nd[c]]);
    }
    for (int i = 0; i < 3; ++i) {
        UD[b][i].d[i] = (T)k.am;
        U[b][i].d[i] = (T)k.c;
    }
    P[b].d[3] = (T)k.c;
    D4<T> Rm[4][3], Rp[4];
    tet_rows<D4<T>>(k, g, UD, U, P, UT, Rm, Rp);
    for (int a = 0; a < 4; ++a) {
        T *o = Ke + 16LL * (16LL * e + 4 * a + b);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 4; ++j) o[4 * i + j] = Rm[a][i].d[j];
        for (int j = 0; j < 4; ++j) o[12 + j] = Rp[a].d[j];
    }
}

template <typename T>
__global__ void k_tan_tri(int Tn, const double *X, const int *tris, const double *v, VmsConst k, T *Kf) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= 3LL * Tn) return;
    const int t = (int)(tid / 3), b = (int)(tid % 3);
    int nd[3];
    for (int a = 0; a < 3; ++a) nd[a] = tris[3LL * t + a];
    D4<T> U[3][3], Rm[3][3];
    for (int c = 0; c < 3; ++c)
        for (int i = 0; i < 3; ++i) U[c][i] = Num<D4<T>>::cst((T)v[3LL * nd[c] + i]);
    for (int i = 0; i < 3; ++i) U[b][i].d[i] = (T)k.c;
    tri_rows<D4<T>>(k, X, nd, U, Rm);
    for (int a = 0; a < 3; ++a) {
        T *o = Kf + 9LL * (9LL * t + 3 * a + b);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) o[3 * i + j] = Rm[a][i].d[j];
    }
}

// Pattern slot s (row A, column B): sum of its tet blocks (ascending e) and
// triangle blocks (ascending t), then the Dirichlet rules: A keeps only the
// diagonal entries of Dirichlet rows/columns, B rows and C columns of
// Dirichlet nodes are zero.
template <typename T>
__global__ void k_tan_gather(long long nnz, const int *slot_row, const int *col, const int *sl_ptr, const int *sl_src,
                             const int *fl_ptr, const int *fl_src, const T *Ke, const T *Kf, const uint8_t *dir,
                             double *Av, double *Bv, double *Cv, double *Dv) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nnz) return;
    double acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0;
    for (int j = sl_ptr[s]; j < sl_ptr[s + 1]; ++j) {
        const T *o = Ke + 16LL * sl_src[j];
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] += (double)o[q];
    }
    for (int j = fl_ptr[s]; j < fl_ptr[s + 1]; ++j) {
        const T *o = Kf + 9LL * fl_src[j];
        for (int i = 0; i < 3; ++i)
            for (int jj = 0; jj < 3; ++jj) acc[4 * i + jj] += (double)o[3 * i + jj];
    }
    const int A = slot_row[s], Bn = col[s];
    const bool dA = dir[A] != 0, dB = dir[Bn] != 0;
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
            const bool keep = (A == Bn && i == j) || (!dA && !dB);
            Av[9 * s + 3 * i + j] = keep ? acc[4 * i + j] : 0.0;
        }
        Bv[3 * s + i] = dA ? 0.0 : acc[4 * i + 3];
        Cv[3 * s + i] = dB ? 0.0 : acc[12 + i];
    }
    Dv[s] = acc[15];
}

// ------------------------------------------------------------------ launchers
void vms_residual(const VmsDev &m, const VmsConst &k, const double *vd, const double *v, const double *p,
                  const double *vtau, int n_out, const int *lr_rp, const int *lr_k, const int *lr_c,
                  const double *lr_v, const double *P, double *R, cudaStream_t s) {
    const double *vt = vtau ? vtau : v;
    if (m.E > 0) {
        k_res_tet<<<(m.E + 127) / 128, 128, 0, s>>>(m.E, m.X, m.tets, vd, v, p, vt, k, m.Re);
        NBP_LAUNCHED();
    }
    if (m.T > 0) {
        k_res_tri<<<(m.T + 127) / 128, 128, 0, s>>>(m.T, m.X, m.tris, v, k, m.Rf);
        NBP_LAUNCHED();
    }
    k_res_gather<<<(m.N + 255) / 256, 256, 0, s>>>(m.N, m.n2t_ptr, m.n2t, m.n2f_ptr, m.n2f, m.Re, m.Rf,
                                                    n_out > 0 ? lr_rp : nullptr, lr_k, lr_c, lr_v,
                                                    n_out > 0 ? P : nullptr, m.dir, R);
    NBP_LAUNCHED();
}

template <typename T>
static void tangent_t(const VmsDev &m, const VmsConst &k, const double *vd, const double *v, const double *p,
                      const double *vt, double *A, double *B, double *C, double *D, cudaStream_t s) {
    T *Ke = (T *)m.Ke, *Kf = (T *)m.Kf;
    if (m.E > 0) {
        k_tan_tet<T><<<(unsigned)((4LL * m.E + 127) / 128), 128, 0, s>>>(m.E, m.X, m.tets, vd, v, p, vt, k, Ke);
        NBP_LAUNCHED();
    }
    if (m.T > 0) {
        k_tan_tri<T><<<(unsigned)((3LL * m.T + 127) / 128), 128, 0, s>>>(m.T, m.X, m.tris, v, k, Kf);
        NBP_LAUNCHED();
    }
    if (m.nnz > 0) {
        k_tan_gather<T><<<(unsigned)((m.nnz + 255) / 256), 256, 0, s>>>(m.nnz, m.slot_row, m.col, m.sl_ptr, m.sl_src,
                                                                        m.fl_ptr, m.fl_src, Ke, Kf, m.dir, A, B, C, D);
        NBP_LAUNCHED();
    }
}

void vms_tangent(const VmsDev &m, const VmsConst &k, const double *vd, const double *v, const double *p,
                 const double *vtau, double *A, double *B, double *C, double *D, cudaStream_t s) {
    const double *vt = vtau ? vtau : v;
    if (m.tangent_fp32) tangent_t<float>(m, k, vd, v, p, vt, A, B, C, D, s);
    else tangent_t<double>(m, k, vd, v, p, vt, A, B, C, D, s);
}

}  // namespace nbp
