// vms.cuh -- on-device assembly of the residual and the consistent tangent
// of the P1-P1 residual-based VMS / generalized-alpha discretisation (paper
// Sec. 2.3-2.5), declarations shared by vms.cu and the C ABI in solver.cu.
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

namespace nbp {

// Physical constants and generalized-alpha coefficients of the assembly.
struct VmsConst {
    double rho, mu, dt, beta, CI, CT;
    double am, af, gm;   // alpha_m, alpha_f, gamma (Sec. 2.4.1)
    double c;            // alpha_f gamma dt
};

// Device copy of the mesh and of the gather maps built at creation.  Scratch
// layout: tet e, local row la, local column lb -> contribution 16 e + 4 la +
// lb (16 values each: the 4x4 block [[A 3x3, B 3], [C 3, D]] row-major);
// outlet triangle t: 9 t + 3 la + lb (a 3x3 velocity block).  Residual
// scratch: 16 e + 4 la + q (q = 3 is the continuity row); 9 t + 3 la + i.
struct VmsDev {
    int N = 0, E = 0, T = 0;
    long long nnz = 0;
    double *X = nullptr;                  // 3N coordinates
    int *tets = nullptr, *tris = nullptr; // 4E, 3T node ids
    uint8_t *dir = nullptr;               // N Dirichlet flags
    int *n2t_ptr = nullptr, *n2t = nullptr;   // node -> 4 e + la, ascending e
    int *n2f_ptr = nullptr, *n2f = nullptr;   // node -> 3 t + la, ascending t
    int *sl_ptr = nullptr, *sl_src = nullptr; // pattern slot -> tet contributions, ascending e
    int *fl_ptr = nullptr, *fl_src = nullptr; // pattern slot -> triangle contributions, ascending t
    int *slot_row = nullptr;              // pattern slot -> row node
    const int *col = nullptr;             // the solver's pattern columns (not owned)
    double *Re = nullptr, *Rf = nullptr;  // residual scratch (16 E, 9 T)
    void *Ke = nullptr, *Kf = nullptr;    // tangent scratch (16 * 16 E, 9 * 9 T) in the tangent's type
    int tangent_fp32 = 1;
};

void vms_residual(const VmsDev &m, const VmsConst &k, const double *vd, const double *v, const double *p,
                  const double *vtau, int n_out, const int *lr_rp, const int *lr_k, const int *lr_c,
                  const double *lr_v, const double *P, double *R, cudaStream_t s);
void vms_tangent(const VmsDev &m, const VmsConst &k, const double *vd, const double *v, const double *p,
                 const double *vtau, double *A, double *B, double *C, double *D, cudaStream_t s);

}  // namespace nbp
