// rcr.cu -- RCR (three-element Windkessel) outlets on the device (paper
// Sec. 2.1, Algorithm 1 and Sec. 2.5): one time step of every outlet's
// distal-pressure ODE, the difference-quotient stiffness m^k that weights
// the outlet's rank-one term in A, and the flow rates Q^k = a^k . v that
// drive them.  One thread per outlet: even 772 outlets are one block of
// work, so the step costs a launch, not bandwidth.
#include "kernels.cuh"
#include "rcr.cuh"

namespace nbp {

// dPi/dt of the RCR circuit: -Pi / (R_d C) + Q / C
__device__ __forceinline__ double rcr_rate(double pi, double q, double Rd, double C) { return -pi / (Rd * C) + q / C; }

// P_{n+1} for the flow q1 at t_{n+1}: n_ts steps of the four-stage scheme
// of Algorithm 1 (stage flows at 1/3 and 2/3 of each substep from the
// linear flow history, weights 1/8, 3/8, 3/8, 1/8); *pi_end = Pi_{n+1}
__device__ double rcr_advance(double Rp, double C, double Rd, double Pd, double pi0, double q0, double q1, double dt,
                              int nts, double *pi_end) {
    const double h = dt / nts;
    double pi = pi0;
    for (int s = 0; s < nts; ++s) {
        const double fa = (double)s / nts, fb = (double)(s + 1) / nts;
        const double qa = (1.0 - fa) * q0 + fa * q1;   // flow at the substep's start
        const double qb = (1.0 - fb) * q0 + fb * q1;   // ... and end
        const double k1 = rcr_rate(pi, qa, Rd, C);
        const double k2 = rcr_rate(pi + k1 * h / 3.0, 2.0 * qa / 3.0 + qb / 3.0, Rd, C);
        const double k3 = rcr_rate(pi - k1 * h / 3.0 + k2 * h, qa / 3.0 + 2.0 * qb / 3.0, Rd, C);
        const double k4 = rcr_rate(pi + k1 * h - k2 * h + k3 * h, qb, Rd, C);
        pi = pi + k1 * h / 8.0 + 3.0 * k2 * h / 8.0 + 3.0 * k3 * h / 8.0 + k4 * h / 8.0;
    }
    *pi_end = pi;
    return Rp * q1 + pi + Pd;
}

__global__ void k_rcr_step(int n_out, nbp_rcr p, const double *__restrict__ Q1, double dt, int nts, double *P1,
                           double *Pi1, double *m, double *r_out, double scale, int *bad) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_out) return;
    const double Rp = p.Rp[k], C = p.C[k], Rd = p.Rd[k], Pd = p.Pd[k], pi0 = p.Pi_n[k], q0 = p.Q_n[k], q1 = Q1[k];
    double pi_end, unused;
    const double P = rcr_advance(Rp, C, Rd, Pd, pi0, q0, q1, dt, nts, &pi_end);
    // m^k = dP_{n+1}/dQ_{n+1} by the central difference of Sec. 2.5
    const double eps = fmax(p.eps_abs, p.eps_rel * fabs(q1));
    const double Pp = rcr_advance(Rp, C, Rd, Pd, pi0, q0, q1 + eps / 2.0, dt, nts, &unused);
    const double Pm = rcr_advance(Rp, C, Rd, Pd, pi0, q0, q1 - eps / 2.0, dt, nts, &unused);
    const double mk = (Pp - Pm) / eps;
    if (P1) P1[k] = P;
    if (Pi1) Pi1[k] = pi_end;
    if (m) m[k] = mk;
    if (r_out) r_out[k] = scale * mk;
    if (bad && !isfinite(mk)) *bad = 1;
}

// Q[k] = a^k . v: lanes stride over the outlet's entries, then a warp tree
// and the warps in order
__global__ void k_outlet_flows(const int *__restrict__ optr, const int *__restrict__ oidx,
                               const double *__restrict__ oval, const double *__restrict__ v, double *__restrict__ Q) {
    __shared__ double red[8];
    const int k = blockIdx.x;
    double s = 0.0;
    for (int q = optr[k] + threadIdx.x; q < optr[k + 1]; q += blockDim.x) s += oval[q] * v[oidx[q]];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        Q[k] = t;
    }
}

void launch_outlet_flows(int n_out, const int *optr, const int *oidx, const double *oval, const double *v, double *Q,
                         cudaStream_t s) {
    if (n_out <= 0) return;
    k_outlet_flows<<<n_out, 256, 0, s>>>(optr, oidx, oval, v, Q);
    NBP_LAUNCHED();
}

void launch_rcr_step(int n_out, const nbp_rcr &p, const double *Q1, double dt, int nts, double *P1, double *Pi1,
                     double *m, double *r_out, double scale, int *bad, cudaStream_t s) {
    if (n_out <= 0) return;
    k_rcr_step<<<(n_out + 127) / 128, 128, 0, s>>>(n_out, p, Q1, dt, nts, P1, Pi1, m, r_out, scale, bad);
    NBP_LAUNCHED();
}

bool rcr_params_ok(const nbp_rcr *p) {
    return p && p->Rp && p->C && p->Rd && p->Pd && p->Pi_n && p->Q_n && p->eps_abs >= 0.0 && p->eps_rel >= 0.0 &&
           (p->eps_abs > 0.0 || p->eps_rel > 0.0);
}

}  // namespace nbp

extern "C" nbp_status nbp_rcr_step(int32_t n_out, const nbp_rcr *p, const double *Q_np1, double dt, int32_t nts,
                                   double *P_np1, double *Pi_np1, double *m, void *stream) {
    using namespace nbp;
    if (n_out < 0 || nts < 1 || !(dt > 0.0)) return NBP_ERR_INVALID;
    if (n_out == 0) return NBP_OK;
    if (!rcr_params_ok(p) || !Q_np1) return NBP_ERR_INVALID;
    try {
        launch_rcr_step(n_out, *p, Q_np1, dt, nts, P_np1, Pi_np1, m, nullptr, 0.0, nullptr, (cudaStream_t)stream);
    } catch (const Error &e) {
        return e.st;
    }
    return NBP_OK;
}
