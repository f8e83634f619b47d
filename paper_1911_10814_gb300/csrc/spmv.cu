// spmv.cu -- instantiation and dispatch of the block-sparse product kernels
// (A: 3x3, B: 3x1, C: 1x3, D / S_hat: 1x1 blocks) for FP64, FP32 and BF16
// values, FP64 or FP32 vectors, and the fused epilogues.
#include "kernels.cuh"
#include "spmv.cuh"

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

namespace nbp {

template <int BR, int BC, int G, typename VT, typename XT>
static void launch_epi(const SpmvArgs &a, int epi, bool lr, cudaStream_t s) {
    const long long threads = (long long)a.nbr * G;
    const unsigned grid = grid_exact(threads);
    switch (epi) {
    case EPI_SET:
        if constexpr (BR == 3 && BC == 3) {
            if (lr) { k_bspmv<BR, BC, G, VT, XT, EPI_SET, true><<<grid, 256, 0, s>>>(a); break; }
        }
        k_bspmv<BR, BC, G, VT, XT, EPI_SET, false><<<grid, 256, 0, s>>>(a);
        break;
    case EPI_ADD: k_bspmv<BR, BC, G, VT, XT, EPI_ADD, false><<<grid, 256, 0, s>>>(a); break;
    case EPI_SUB: k_bspmv<BR, BC, G, VT, XT, EPI_SUB, false><<<grid, 256, 0, s>>>(a); break;
    case EPI_RES:
        if constexpr (BR == BC) { k_bspmv<BR, BC, G, VT, XT, EPI_RES, false><<<grid, 256, 0, s>>>(a); break; }
        throw Error{NBP_ERR_INVALID, "spmv: residual epilogue needs square blocks"};
    case EPI_CHEB:
        if constexpr (BR == BC) { k_bspmv<BR, BC, G, VT, XT, EPI_CHEB, false><<<grid, 256, 0, s>>>(a); break; }
        throw Error{NBP_ERR_INVALID, "spmv: Chebyshev epilogue needs square blocks"};
    default: throw Error{NBP_ERR_INVALID, "spmv: unknown epilogue"};
    }
    NBP_LAUNCHED();
}

template <int BR, int BC, typename VT, typename XT>
static void launch_g(const SpmvArgs &a, int G, int epi, bool lr, cudaStream_t s) {
    if constexpr (BR == BC) {
        switch (G) {
        case 4: launch_epi<BR, BC, 4, VT, XT>(a, epi, lr, s); return;
        case 8: launch_epi<BR, BC, 8, VT, XT>(a, epi, lr, s); return;
        case 16: launch_epi<BR, BC, 16, VT, XT>(a, epi, lr, s); return;
        default: launch_epi<BR, BC, 32, VT, XT>(a, epi, lr, s); return;
        }
    } else {
        launch_epi<BR, BC, 8, VT, XT>(a, epi, lr, s);
    }
}

template <int BR, int BC, typename XT>
static void launch_vt(const DMat &M, int vsel, SpmvArgs a, int G, int epi, bool lr, cudaStream_t s) {
    if constexpr (sizeof(XT) == 8) {
        require(vsel == 0, NBP_ERR_INVALID, "spmv: FP64 vectors need FP64 values");
        a.val = M.v;
        launch_g<BR, BC, double, double>(a, G, epi, lr, s);
    } else {
        if (vsel == 2) {
            require(M.v16 != nullptr, NBP_ERR_STATE, "spmv: BF16 values not built (run setup with precision 2)");
            a.val = M.v16;
            launch_g<BR, BC, __nv_bfloat16, float>(a, G, epi, lr, s);
        } else {
            require(M.v32 != nullptr, NBP_ERR_STATE, "spmv: FP32 values not built (run setup with precision >= 1)");
            a.val = M.v32;
            launch_g<BR, BC, float, float>(a, G, epi, lr, s);
        }
    }
}

int choose_group(const DMat &M) {
    const double per_row = M.nbr ? (double)M.nnz * M.bb() / M.nbr : 0.0;
    if (per_row <= 10) return 4;
    if (per_row <= 40) return 8;
    if (per_row <= 160) return 16;
    return 32;
}

template <int BS, typename VT, typename XT, int C>
static void launch_sell_epi(const SpmvArgs &a, int epi, bool lr, cudaStream_t s) {
    const unsigned grid = grid_exact((long long)a.nslice * C);
    switch (epi) {
    case EPI_SET:
        if constexpr (BS == 3) {
            if (lr) { k_sell<BS, VT, XT, EPI_SET, true, C><<<grid, 256, 0, s>>>(a); break; }
        }
        k_sell<BS, VT, XT, EPI_SET, false, C><<<grid, 256, 0, s>>>(a);
        break;
    case EPI_ADD: k_sell<BS, VT, XT, EPI_ADD, false, C><<<grid, 256, 0, s>>>(a); break;
    case EPI_SUB: k_sell<BS, VT, XT, EPI_SUB, false, C><<<grid, 256, 0, s>>>(a); break;
    case EPI_RES: k_sell<BS, VT, XT, EPI_RES, false, C><<<grid, 256, 0, s>>>(a); break;
    case EPI_CHEB: k_sell<BS, VT, XT, EPI_CHEB, false, C><<<grid, 256, 0, s>>>(a); break;
    default: throw Error{NBP_ERR_INVALID, "spmv: unknown epilogue"};
    }
    NBP_LAUNCHED();
}

template <int BS, typename VT, typename XT, int C, int T>
static void launch_sellm_epi(const SpmvArgs &a, int epi, cudaStream_t s) {
    const unsigned grid = grid_exact((long long)a.nslice * C * T);
    switch (epi) {
    case EPI_SET: k_sellm<BS, VT, XT, EPI_SET, C, T><<<grid, 256, 0, s>>>(a); break;
    case EPI_ADD: k_sellm<BS, VT, XT, EPI_ADD, C, T><<<grid, 256, 0, s>>>(a); break;
    case EPI_SUB: k_sellm<BS, VT, XT, EPI_SUB, C, T><<<grid, 256, 0, s>>>(a); break;
    case EPI_RES: k_sellm<BS, VT, XT, EPI_RES, C, T><<<grid, 256, 0, s>>>(a); break;
    case EPI_CHEB: k_sellm<BS, VT, XT, EPI_CHEB, C, T><<<grid, 256, 0, s>>>(a); break;
    default: throw Error{NBP_ERR_INVALID, "spmv: unknown epilogue"};
    }
    NBP_LAUNCHED();
}

template <int BS, typename VT, typename XT, int C>
static void launch_sellm_t(const SpmvArgs &a, int epi, cudaStream_t s, int T) {
    if (T == 8) launch_sellm_epi<BS, VT, XT, C, 8>(a, epi, s);
    else if (T == 4) launch_sellm_epi<BS, VT, XT, C, 4>(a, epi, s);
    else launch_sellm_epi<BS, VT, XT, C, 2>(a, epi, s);
}

// T threads per row (T = 1: the one-thread kernel, which also has the
// rank-one epilogue)
template <int BS, typename VT, typename XT>
static void launch_sell_c(const DMat &M, const SpmvArgs &a, int epi, bool lr, cudaStream_t s, int T) {
    if (T > 1 && !lr) {
        if (M.sl_c == 8) launch_sellm_t<BS, VT, XT, 8>(a, epi, s, T);
        else launch_sellm_t<BS, VT, XT, 32>(a, epi, s, T);
        return;
    }
    if (M.sl_c == 8) launch_sell_epi<BS, VT, XT, 8>(a, epi, lr, s);
    else launch_sell_epi<BS, VT, XT, 32>(a, epi, lr, s);
}

template <int BS, typename XT>
static void launch_sell(const DMat &M, int vsel, SpmvArgs a, int epi, bool lr, cudaStream_t s, int T) {
    a.nslice = M.nslice;
    a.sl_ptr = M.sl_ptr;
    a.sl_ci = M.sl_ci;
    if constexpr (sizeof(XT) == 8) {
        a.val = M.sl_v;
        launch_sell_c<BS, double, double>(M, a, epi, lr, s, T);
    } else if (vsel == 2) {
        require(M.sl_v16 != nullptr, NBP_ERR_STATE, "spmv: BF16 sliced values not built");
        a.sl_ptr = M.sl2_ptr;   // paired layout
        a.sl_ci = M.sl2_ci;
        a.val = M.sl_v16;
        launch_sell_c<BS, __nv_bfloat16, float>(M, a, epi, lr, s, T);
    } else {
        require(M.sl_v32 != nullptr, NBP_ERR_STATE, "spmv: FP32 sliced values not built");
        a.val = M.sl_v32;
        launch_sell_c<BS, float, float>(M, a, epi, lr, s, T);
    }
}

template <int BR, int BC, typename VT, typename XT, int C>
static void launch_sellr_epi(const SpmvArgs &a, int epi, cudaStream_t s) {
    const unsigned grid = grid_exact((long long)a.nslice * C);
    switch (epi) {
    case EPI_SET: k_sellr<BR, BC, VT, XT, EPI_SET, C><<<grid, 256, 0, s>>>(a); break;
    case EPI_ADD: k_sellr<BR, BC, VT, XT, EPI_ADD, C><<<grid, 256, 0, s>>>(a); break;
    case EPI_SUB: k_sellr<BR, BC, VT, XT, EPI_SUB, C><<<grid, 256, 0, s>>>(a); break;
    default: throw Error{NBP_ERR_INVALID, "spmv: rectangular blocks take SET, ADD or SUB"};
    }
    NBP_LAUNCHED();
}

// rectangular blocks (3x1, 1x3) on their sliced-ELL copy, FP64 or FP32 values
template <int BR, int BC, typename XT>
static void launch_sellr(const DMat &M, int vsel, SpmvArgs a, int epi, cudaStream_t s) {
    a.nslice = M.nslice;
    a.sl_ptr = M.sl_ptr;
    a.sl_ci = M.sl_ci;
    if constexpr (sizeof(XT) == 8) {
        a.val = M.sl_v;
        if (M.sl_c == 8) launch_sellr_epi<BR, BC, double, double, 8>(a, epi, s);
        else launch_sellr_epi<BR, BC, double, double, 32>(a, epi, s);
    } else {
        a.val = M.sl_v32;
        if (M.sl_c == 8) launch_sellr_epi<BR, BC, float, float, 8>(a, epi, s);
        else launch_sellr_epi<BR, BC, float, float, 32>(a, epi, s);
    }
}

// Algorithmic bytes of one product y = epilogue(M x): every stored block's
// values and column index once, the row pointers (flat kernel) or the slice
// pointers (sliced layouts; their padding is not counted), x once, and the
// epilogue's vectors: SET writes y; ADD and SUB read and write y; RES reads
// b and writes y; CHEB reads b, d and the block-diagonal inverse and writes
// d and xout (x_i itself is the product's input, counted once).
static double product_bytes(const DMat &M, int vsel, int xs, int epi, bool sliced) {
    const double vb = xs == 8 ? 8.0 : (vsel == 2 ? 2.0 : 4.0);
    double b = (double)M.nnz * (M.bb() * vb + 4.0);
    b += sliced ? (double)(M.nslice + 1) * 8.0 : (double)(M.nbr + 1) * 4.0;
    const double nx = (double)M.nbc * M.bc * xs, ny = (double)M.nbr * M.br * xs;
    b += nx;
    if (epi == EPI_SET) b += ny;
    else if (epi == EPI_CHEB) b += 4.0 * ny + (double)M.nbr * M.br * M.br * xs;
    else b += 2.0 * ny;
    return b;
}

static int sell_threads(const DMat &M) {
    const int G = M.tuned >= 0 ? M.tuned : 0;
    return G == 0 ? 1 : (is_sellm(G) ? G - kSellMT : 0);
}

bool spmv_dot_ok(const DMat &M, int vsel, int xbytes, long long max_blocks) {
    if (M.br != 1 || M.bc != 1 || !M.sl_ci || M.nbr == 0) return false;
    const int T = sell_threads(M);
    if (T == 0) return false;
    if (((long long)M.nslice * M.sl_c * T + 255) / 256 > max_blocks) return false;
    if (xbytes == 8) return M.sl_v != nullptr;
    return vsel == 2 ? M.sl_v16 != nullptr : M.sl_v32 != nullptr;
}

template <typename VT, typename XT, int C>
static void launch_sell_dot(const SpmvArgs &a, const DotArgs &q, int T, cudaStream_t s) {
    const unsigned grid = grid_exact((long long)a.nslice * C * T);
    if (T == 8) k_sell_dot<VT, XT, C, 8><<<grid, 256, 0, s>>>(a, q);
    else if (T == 4) k_sell_dot<VT, XT, C, 4><<<grid, 256, 0, s>>>(a, q);
    else if (T == 2) k_sell_dot<VT, XT, C, 2><<<grid, 256, 0, s>>>(a, q);
    else k_sell_dot<VT, XT, C, 1><<<grid, 256, 0, s>>>(a, q);
    NBP_LAUNCHED();
}
template <typename VT, typename XT>
static void launch_sell_dot_c(const DMat &M, const SpmvArgs &a, const DotArgs &q, int T, cudaStream_t s) {
    if (M.sl_c == 8) launch_sell_dot<VT, XT, 8>(a, q, T, s);
    else launch_sell_dot<VT, XT, 32>(a, q, T, s);
}

template <typename XT>
double spmv_dot(const DMat &M, int vsel, SpmvArgs a, const DotArgs &q, cudaStream_t s) {
    const int T = sell_threads(M);
    a.nbr = M.nbr;
    a.nslice = M.nslice;
    a.sl_ptr = M.sl_ptr;
    a.sl_ci = M.sl_ci;
    if constexpr (sizeof(XT) == 8) {
        a.val = M.sl_v;
        launch_sell_dot_c<double, double>(M, a, q, T, s);
    } else if (vsel == 2) {
        a.sl_ptr = M.sl2_ptr;   // paired layout
        a.sl_ci = M.sl2_ci;
        a.val = M.sl_v16;
        launch_sell_dot_c<__nv_bfloat16, float>(M, a, q, T, s);
    } else {
        a.val = M.sl_v32;
        launch_sell_dot_c<float, float>(M, a, q, T, s);
    }
    const double ny = (double)M.nbr * sizeof(XT);
    return product_bytes(M, vsel, (int)sizeof(XT), EPI_SET, true) + (q.da != a.y ? ny : 0.0) + (q.db ? ny : 0.0);
}

template <typename XT>
double spmv(const DMat &M, int vsel, SpmvArgs a, int epi, bool lr, cudaStream_t s, int G) {
    a.nbr = M.nbr;
    a.rp = M.rp;
    a.ci = M.ci;
    if (a.nbr == 0) return 0.0;
    constexpr int xs = (int)sizeof(XT);
    // rectangular coupling blocks: sliced ELL for FP64 / FP32 values (BF16: flat kernel)
    if (M.br != M.bc && M.sl_ci && G <= 0 && epi <= EPI_SUB && vsel != 2 &&
        (sizeof(XT) == 8 ? M.sl_v != nullptr : M.sl_v32 != nullptr)) {
        if (M.br == 3 && M.bc == 1) { launch_sellr<3, 1, XT>(M, vsel, a, epi, s); return product_bytes(M, vsel, xs, epi, true); }
        if (M.br == 1 && M.bc == 3) { launch_sellr<1, 3, XT>(M, vsel, a, epi, s); return product_bytes(M, vsel, xs, epi, true); }
    }
    const bool sell_ok = M.sl_ci && M.br == M.bc && (sizeof(XT) == 8 ? M.sl_v != nullptr : true);
    if (G < 0) G = (M.tuned >= 0) ? M.tuned : (sell_ok ? 0 : choose_group(M));
    if ((G == 0 || is_sellm(G)) && !sell_ok) G = choose_group(M);
    if (sell_ok && (G == 0 || is_sellm(G))) {
        const int T = G == 0 ? 1 : G - kSellMT;
        if (M.br == 3) launch_sell<3, XT>(M, vsel, a, epi, lr, s, T);
        else launch_sell<1, XT>(M, vsel, a, epi, lr, s, T);
        return product_bytes(M, vsel, xs, epi, true);
    }
    if (M.br == 3 && M.bc == 3) launch_vt<3, 3, XT>(M, vsel, a, G, epi, lr, s);
    else if (M.br == 3 && M.bc == 1) launch_vt<3, 1, XT>(M, vsel, a, G, epi, lr, s);
    else if (M.br == 1 && M.bc == 3) launch_vt<1, 3, XT>(M, vsel, a, G, epi, lr, s);
    else if (M.br == 1 && M.bc == 1) launch_vt<1, 1, XT>(M, vsel, a, G, epi, lr, s);
    else throw Error{NBP_ERR_INVALID, "spmv: unsupported block shape"};
    return product_bytes(M, vsel, xs, epi, false);
}

template double spmv<double>(const DMat &, int, SpmvArgs, int, bool, cudaStream_t, int);
template double spmv<float>(const DMat &, int, SpmvArgs, int, bool, cudaStream_t, int);
template double spmv_dot<double>(const DMat &, int, SpmvArgs, const DotArgs &, cudaStream_t);
template double spmv_dot<float>(const DMat &, int, SpmvArgs, const DotArgs &, cudaStream_t);

}  // namespace nbp
