// rcr.cuh -- launchers of the RCR outlet kernels (rcr.cu), for the context
// entry points in solver.cu.  Internal header.
#pragma once
#include "nbp_common.cuh"

namespace nbp {

// Q[k] = a^k . v for the n_out sparse outlet vectors (optr/oidx/oval), one
// block per outlet, fixed-order reduction
void launch_outlet_flows(int n_out, const int *optr, const int *oidx, const double *oval, const double *v, double *Q,
                         cudaStream_t s);

// One RCR step per outlet (see nbp_rcr_step); r_out (optional) gets
// scale * m^k, bad (optional) is set to 1 when some m^k is not finite
void launch_rcr_step(int n_out, const nbp_rcr &p, const double *Q1, double dt, int nts, double *P1, double *Pi1,
                     double *m, double *r_out, double scale, int *bad, cudaStream_t s);

// parameter block complete (every array set, a positive difference step)
bool rcr_params_ok(const nbp_rcr *p);

}  // namespace nbp
