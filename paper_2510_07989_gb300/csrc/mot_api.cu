// C ABI of the GB300 MOT library: handle lifetime, topology, operator upload,
// the MOT step pipeline and the batched GMRES solve of Q_0 (paper Eq. (MOT)).
//
// Step i (all on one stream, FP64):
//   rho1, rho2                   <- incident field tested (Section V-C)
//   s1, s2                       <- block-sparse history over lags 1..K
//   b = LF(rho1 - s1, rho2 - s2), LF(y1, y2) = T^{SH} G^-1 y1 + T^L G^-1 P^{LH} y2
//   w_i = GMRES(Q_0, b),  Q_0 w = LF(A_0 l + A^_0 s, A~_0 l + A_0 s),
//         s = P^S w, l = w - s   (Section V-B product form, no dense Q_k)
//   ring slot <- variants of l_i, s_i; currents and Fourier sums (Eq. (dis_jm))
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <tuple>
#include <numeric>
#include <string>
#include <condition_variable>
#include <mutex>
#include <thread>
#include <vector>

#include "mot_internal.h"

#define MOT_API extern "C" __attribute__((visibility("default")))

namespace mot {

int fail(mot_handle* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    return code;
}

int cuda_fail(mot_handle* h, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    if (h) h->err = m;
    return e == cudaErrorMemoryAllocation ? MOT_EOOM : MOT_ECUDA;
}

void* dalloc(mot_handle* h, size_t bytes) {
    void* p = nullptr;
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    // Zeroed before returning: the memory may next be used from a non-blocking
    // stream (mot_run_many), which is not ordered after the legacy stream that
    // cudaMemset runs on, and cudaMemset may return before it has run.
    if (cudaMemset(p, 0, bytes) != cudaSuccess || cudaStreamSynchronize(nullptr) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(p);
        return nullptr;
    }
    h->device_bytes += (int64_t)bytes;
    return p;
}

// mixed-precision kernels (k_mixed.cu)
void launch_history32(mot_handle* h, const TaskList& tl, const float* tiles, const float* ring, const float* win,
                      const float* kry, int mode, long long step_i, double* out_s1, double* out_s2, cudaStream_t s);
void launch_sgemm_d(mot_handle* h, int M, int N, int K, const float* A, const float* X, double* Y, cudaStream_t s);
void launch_d2f(mot_handle* h, size_t n, const double* x, float* y, cudaStream_t s);
void launch_unit_cols(mot_handle* h, long long J0, long long Jend, double* X, cudaStream_t s);
void launch_scatter_cols(mot_handle* h, long long J0, long long Jend, const double* Y, double* D, long long ldd,
                         cudaStream_t s);
void launch_unit_lf(mot_handle* h, long long Q0, long long Qend, double* y1, double* y2, cudaStream_t s);
void launch_scatter_lf(mot_handle* h, long long Q0, long long Qend, const double* out, double* D, long long ldd,
                       cudaStream_t s);

// dense factorisation (k_dense.cu)
int dense_lu(mot_handle* h, int n, double* A, int* piv, int* d_bad, cudaStream_t s);
void dense_pad_identity(mot_handle* h, int n, int ne, double* A, cudaStream_t s);
void dense_lap_plus_j(mot_handle* h, const DCsr& L, int npd, double* A, cudaStream_t s);
int pcg_dense_prec(mot_handle* h, const DCsr& L, int npd, const float* M, const double* f, int C, double* z,
                   double* work, double* d_scal, float* fstage, double tol, int maxit, cudaStream_t s);
void dense_inverse_from_lu(mot_handle* h, int n, const double* LU, const int* piv, double* X, cudaStream_t s);
void direct_laplacian_solve(mot_handle* h, int N, int npd, const double* Linv, const double* f, int C, double* r,
                            double* z, double* sc, cudaStream_t s);

// extra launch wrappers (k_linalg.cu)
void launch_pack2(mot_handle* h, const double* a, const double* b, int C, double* out, cudaStream_t s);
void launch_unpack_q(mot_handle* h, const double* X, const double* P, int C, double* q1, double* q2, cudaStream_t s);
void launch_far_field(mot_handle* h, int n_dir, const double* dirs, double* E, cudaStream_t s);
void launch_pack_cur(mot_handle* h, double* out, cudaStream_t s);

}  // namespace mot

using namespace mot;

#define CK(call)                                                     \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call);       \
    } while (0)
#define CK_H(hh, call)                                               \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail(hh, e_, #call);      \
    } while (0)

namespace {

struct HostCsr {
    int n = 0, m = 0;
    std::vector<int> rp, ci;
    std::vector<double> va;
};

int upload_csr(mot_handle* h, const HostCsr& A, DCsr& D) {
    D.n = A.n;
    D.m = A.m;
    D.nnz = (int64_t)A.ci.size();
    D.rowptr = (int*)dalloc(h, sizeof(int) * (A.n + 1));
    D.col = (int*)dalloc(h, sizeof(int) * std::max<size_t>(1, A.ci.size()));
    D.val = (double*)dalloc(h, sizeof(double) * std::max<size_t>(1, A.va.size()));
    if (!D.rowptr || !D.col || !D.val) return fail(h, MOT_EOOM, "device allocation (CSR)");
    CK(cudaMemcpy(D.rowptr, A.rp.data(), sizeof(int) * (A.n + 1), cudaMemcpyHostToDevice));
    if (!A.ci.empty()) {
        CK(cudaMemcpy(D.col, A.ci.data(), sizeof(int) * A.ci.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(D.val, A.va.data(), sizeof(double) * A.va.size(), cudaMemcpyHostToDevice));
    }
    return MOT_OK;
}

HostCsr csr_from_triplets(int n, int m, std::vector<std::tuple<int, int, double>>& t) {
    std::sort(t.begin(), t.end(), [](const auto& a, const auto& b) {
        return std::get<0>(a) != std::get<0>(b) ? std::get<0>(a) < std::get<0>(b) : std::get<1>(a) < std::get<1>(b);
    });
    HostCsr A;
    A.n = n;
    A.m = m;
    A.rp.assign(n + 1, 0);
    for (size_t i = 0; i < t.size(); i++) {
        int r = std::get<0>(t[i]), c = std::get<1>(t[i]);
        double v = std::get<2>(t[i]);
        if (!A.ci.empty() && A.rp[r + 1] > 0 && (int)A.ci.size() > 0 && i > 0 && std::get<0>(t[i - 1]) == r &&
            std::get<1>(t[i - 1]) == c) {
            A.va.back() += v;
            continue;
        }
        A.ci.push_back(c);
        A.va.push_back(v);
        A.rp[r + 1]++;
    }
    for (int r = 0; r < n; r++) A.rp[r + 1] += A.rp[r];
    return A;
}

uint64_t spread3(uint64_t x) {
    x &= 0x1fffff;
    x = (x | x << 32) & 0x1f00000000ffffULL;
    x = (x | x << 16) & 0x1f0000ff0000ffULL;
    x = (x | x << 8) & 0x100f00f00f00f00fULL;
    x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
    x = (x | x << 2) & 0x1249249249249249ULL;
    return x;
}

// ---------------------------------------------------------------- step pieces
struct Work {
    double *rho1, *rho2, *s1, *s2, *y1, *y2, *b, *x, *w, *r, *sig, *ell, *tmp, *z2;
    double *kry;              // [2][3] block vectors
    double *Y4, *GY4, *X4, *PX4;  // 4B-column block vectors
    double *q1, *q2, *t1, *t2, *dd, *pd;
    double *fvec, *zvec;      // faces / vertices x 4B
    double *cgw;              // CG scratch 4 x maxN x 4B
    double *hc1, *hc2, *hsum, *nrm, *beta, *ygm;
};

Work work_of(mot_handle* h) {
    Work W;
    const size_t bv = (size_t)h->npad * 2 * h->B;
    const size_t bv4 = 2 * bv;
    const int maxN = std::max(std::max(h->npad, h->nf), h->nv);
    double* p = h->d_work;
    auto take = [&](size_t n) {
        double* q = p;
        p += (n + 31) / 32 * 32;
        return q;
    };
    W.rho1 = take(bv);
    W.rho2 = take(bv);
    W.s1 = take(bv);
    W.s2 = take(bv);
    W.y1 = take(bv);
    W.y2 = take(bv);
    W.b = take(bv);
    W.x = take(bv);
    W.w = take(bv);
    W.r = take(bv);
    W.sig = take(bv);
    W.ell = take(bv);
    W.tmp = take(bv);
    W.z2 = take(bv);
    W.kry = take(6 * bv);
    W.Y4 = take(bv4);
    W.GY4 = take(bv4);
    W.X4 = take(bv4);
    W.PX4 = take(bv4);
    W.q1 = take(bv);
    W.q2 = take(bv);
    W.t1 = take(bv);
    W.t2 = take(bv);
    W.dd = take(bv);
    W.pd = take(bv);
    W.fvec = take((size_t)std::max(h->nf, h->nv) * 4 * h->B);
    W.zvec = take((size_t)std::max(h->nf, h->nv) * 4 * h->B);
    W.cgw = take((size_t)4 * maxN * 4 * h->B);
    const size_t gm = (size_t)(h->gm_m + 1) * h->B;
    W.hc1 = take(gm);
    W.hc2 = take(gm);
    W.hsum = take(gm);
    W.nrm = take(h->B);
    W.beta = take(h->B);
    W.ygm = take(gm);
    return W;
}

size_t work_doubles(mot_handle* h) {
    const size_t bv = (size_t)h->npad * 2 * h->B;
    const int maxN = std::max(std::max(h->npad, h->nf), h->nv);
    const size_t gm = (size_t)(h->gm_m + 1) * h->B;
    size_t n = 0;
    auto add = [&](size_t k) { n += (k + 31) / 32 * 32; };
    for (int i = 0; i < 14; i++) add(bv);
    add(6 * bv);
    for (int i = 0; i < 4; i++) add(2 * bv);
    for (int i = 0; i < 6; i++) add(bv);
    add((size_t)std::max(h->nf, h->nv) * 4 * h->B);
    add((size_t)std::max(h->nf, h->nv) * 4 * h->B);
    add((size_t)4 * maxN * 4 * h->B);
    add(gm);
    add(gm);
    add(gm);
    add(h->B);
    add(h->B);
    add(gm);
    return n;
}

// out = P^Sigma x  (C = 2B columns); Sigma^T x -> CG on Sigma^T Sigma -> Sigma z.
// The mixed path preconditions the FP64 CG with an FP32 dense (L + 11^T/N_f)^{-1}.
void project_sigma(mot_handle* h, const Work& W, const double* x, double* out, cudaStream_t s) {
    const int C = 2 * h->B;
    launch_sigma_t(h, x, C, W.fvec, s);
    if (h->d_Lfinv64) {  // FP64 path with fp64_direct: the dense pseudo-inverse
        direct_laplacian_solve(h, h->nf, h->dfpd, h->d_Lfinv64, W.fvec, C, h->d_dir_r, h->d_dir_z, h->d_dir_sc, s);
        launch_sigma(h, h->d_dir_z, C, out, s);
        return;
    }
    if (h->d_Lfinvf && h->d_pcg_work && !h->precomputing)
        h->last_pcg_iters = pcg_dense_prec(h, h->Lf, h->nfpd, h->d_Lfinvf, W.fvec, C, W.zvec, h->d_pcg_work,
                                           h->d_pcg_scal, h->d_pcg_f32, h->opt.cg_tol, 50, s);
    else
        launch_cg(h, h->Lf, nullptr, W.fvec, C, W.zvec, W.cgw, s);
    launch_sigma(h, W.zvec, C, out, s);
}

// out = P^Lambda x for C columns
void project_lambda(mot_handle* h, const Work& W, const double* x, int C, double* out, cudaStream_t s) {
    launch_lambda_t(h, x, C, W.fvec, s);
    if (h->d_Lvinv64) {  // FP64 path with fp64_direct: the dense pseudo-inverse
        direct_laplacian_solve(h, h->nv, h->dvpd, h->d_Lvinv64, W.fvec, C, h->d_dir_r, h->d_dir_z, h->d_dir_sc, s);
        launch_lambda(h, h->d_dir_z, C, out, s);
        return;
    }
    launch_cg(h, h->Lv, nullptr, W.fvec, C, W.zvec, W.cgw, s);
    launch_lambda(h, W.zvec, C, out, s);
}

// out = T^{SH} G^-1 y1 + T^L G^-1 P^{LH} y2   (Eq. (CP), (reg_DCP_PMCHWT))
void left_factor(mot_handle* h, const Work& W, const double* y1, const double* y2, double* out, cudaStream_t s) {
    const int C = 2 * h->B;
    const int n = h->npad * C;
    project_sigma(h, W, y2, W.tmp, s);
    launch_axpby(h, n, 1.0, y2, -1.0, W.tmp, W.z2, s);  // z2 = P^{LH} y2
    launch_pack2(h, y1, W.z2, C, W.Y4, s);
    if (h->d_Ginv64) {  // FP64 path with fp64_direct: X = G^{-1} Y with the dense inverse
        launch_gemm_rect(h, h->npad, h->npad, h->d_Ginv64, W.Y4, 2 * C, W.X4, s);
    } else {
        launch_spmv(h, h->Gt, W.Y4, 2 * C, W.GY4, s);        // G^T Y
        launch_cg(h, h->G, &h->Gt, W.GY4, 2 * C, W.X4, W.cgw, s);  // (G^T G) X = G^T Y
    }
    project_lambda(h, W, W.X4, 2 * C, W.PX4, s);
    launch_unpack_q(h, W.X4, W.PX4, C, W.q1, W.q2, s);  // q1 = P^{SH} x1, q2 = P^L x2
    launch_gemm(h, h->d_T0s, W.q1, C, W.t1, s);
    launch_gemm(h, h->d_T0h, W.q2, C, W.t2, s);
    launch_axpby(h, n, 1.0, W.t2, -1.0, W.t1, W.dd, s);
    project_lambda(h, W, W.dd, C, W.pd, s);
    launch_axpby(h, n, 1.0, W.t1, 1.0, W.pd, out, s);   // P^{SH} t1 + P^L t2
}

bool mixed(const mot_handle* h) { return h->opt.precision == MOT_PREC_MIXED && h->d_Q0 && !h->precomputing; }
bool mflag(const mot_handle* h, int bit) { return (h->opt.mixed_flags & bit) != 0; }
// emulated products on the tensor cores: requested and an sm_100-family GPU
bool emu_ok(const mot_handle* h) {
    int major = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, h->dev);
    return mflag(h, MOT_MIX_EMU64) && major == 10;
}

// out = Q_0 v with the dense FP64 Q_0 (the refinement residual of the mixed path)
void apply_q0_dense64(mot_handle* h, const double* v, double* out, cudaStream_t s) {
    if (h->emu_Q0.a16)  // emulated FP64 on the tensor cores (MOT_MIX_EMU64)
        launch_emu_gemm(h, h->emu_Q0, v, h->B, out, s);
    else
        launch_gemm_rect(h, 2 * h->npad, 2 * h->npad, h->d_Q0, v, h->B, out, s);
}

// out = Q_0 v: dense Q_0 (mixed path, FP32 or FP64 copy) or the FP64 product form
void apply_q0(mot_handle* h, const Work& W, const double* v, double* out, cudaStream_t s) {
    const int n = h->npad * 2 * h->B;
    const size_t bv = (size_t)n;
    if (mixed(h)) {
        const double* in = v;
        if (h->prec_active) {  // right preconditioning: Q_0 (M v)
            if (h->emu_Minv.a16) {
                launch_emu_gemm(h, h->emu_Minv, v, h->B, W.q1, s);
            } else {
                launch_d2f(h, bv, v, h->d_xf, s);
                launch_sgemm_d(h, 2 * h->npad, h->B, 2 * h->npad, h->d_Minvf, h->d_xf, W.q1, s);
            }
            in = W.q1;
        }
        if (mflag(h, MOT_MIX_Q032)) {
            if (h->emu_Q0s.a16) {
                launch_emu_gemm(h, h->emu_Q0s, in, h->B, out, s);
            } else {
                launch_d2f(h, bv, in, h->d_xf, s);
                launch_sgemm_d(h, 2 * h->npad, h->B, 2 * h->npad, h->d_Q0f, h->d_xf, out, s);
            }
        } else {
            apply_q0_dense64(h, in, out, s);
        }
        return;
    }
    if (h->prec_active && h->d_Minv64) {  // FP64 right preconditioning: Q_0 (M v), M = Q_0^{-1} in FP64
        launch_gemm_rect(h, 2 * h->npad, 2 * h->npad, h->d_Minv64, v, h->B, W.q1, s);
        v = W.q1;  // consumed before left_factor reuses W.q1
    }
    project_sigma(h, W, v, W.sig, s);
    launch_axpby(h, n, 1.0, v, -1.0, W.sig, W.ell, s);
    launch_variants(h, W.ell, W.kry, h->eta, h->etap, s);
    launch_variants(h, W.sig, W.kry + 3 * bv, h->eta, h->etap, s);
    launch_history(h, h->lag0, h->d_tiles, nullptr, nullptr, W.kry, 1, 0, W.y1, W.y2, s);
    left_factor(h, W, W.y1, W.y2, out, s);
}

// GMRES on Q_0 x = b, started from the x passed in (x0 = 0 when have_x0 is
// false); the relative tolerance always refers to |b|.
int gmres(mot_handle* h, const Work& W, const double* b, double* x, bool have_x0, double tol, cudaStream_t s) {
    const int B = h->B;
    const size_t bv = (size_t)h->npad * 2 * B;
    const int m = h->gm_m;
    h->gm_tol = tol;
    launch_gm_norm(h, b, W.beta, s);
    launch_gm_init(h, W.beta, 1, s);  // records |b| as the reference norm
    if (have_x0) {
        apply_q0(h, W, x, W.r, s);
        launch_axpby(h, (int)bv, 1.0, b, -1.0, W.r, W.r, s);
        launch_gm_norm(h, W.r, W.beta, s);
        launch_gm_init(h, W.beta, 0, s);
        launch_gm_scale(h, W.r, W.beta, h->d_V, s);
    } else {
        CK(cudaMemsetAsync(x, 0, sizeof(double) * bv, s));
        launch_gm_scale(h, b, W.beta, h->d_V, s);
    }
    int total = 0;
    bool converged = false;
    std::vector<int> act(B);
    for (int cycle = 0; !converged && total < h->opt.gmres_maxit; cycle++) {
        int jend = 0;
        for (int j = 0; j < m && total < h->opt.gmres_maxit; j++) {
            const double* Vj = h->d_V + (size_t)j * bv;
            apply_q0(h, W, Vj, W.w, s);
            launch_gm_dots(h, h->d_V, j + 1, W.w, W.hc1, s);
            launch_gm_update(h, h->d_V, j + 1, W.hc1, W.w, s);
            launch_gm_dots(h, h->d_V, j + 1, W.w, W.hc2, s);
            launch_gm_update(h, h->d_V, j + 1, W.hc2, W.w, s);
            launch_axpby(h, (j + 1) * B, 1.0, W.hc1, 1.0, W.hc2, W.hsum, s);
            launch_gm_norm(h, W.w, W.nrm, s);
            launch_gm_arnoldi_finish(h, j, W.hsum, W.nrm, s);
            launch_gm_scale(h, W.w, W.nrm, h->d_V + (size_t)(j + 1) * bv, s);
            CK(cudaMemcpyAsync(act.data(), h->d_gm_active, sizeof(int) * B, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            total++;
            jend = j + 1;
            bool any = false;
            for (int k = 0; k < B; k++) any |= act[k] != 0;
            if (!any) {
                converged = true;
                break;
            }
        }
        if (jend > 0) launch_gm_solve_update(h, W.ygm, x, s);
        if (converged || total >= h->opt.gmres_maxit) break;
        // restart from the true residual
        apply_q0(h, W, x, W.r, s);
        launch_axpby(h, (int)bv, 1.0, b, -1.0, W.r, W.r, s);
        launch_gm_norm(h, W.r, W.beta, s);
        launch_gm_init(h, W.beta, 0, s);
        launch_gm_scale(h, W.r, W.beta, h->d_V, s);
    }
    std::vector<double> res(B);
    CK(cudaMemcpyAsync(res.data(), h->d_resid, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    h->last_gmres_iters = total;
    h->last_gmres_resid = 0;
    for (double r : res) h->last_gmres_resid = std::max(h->last_gmres_resid, r);
    return converged ? MOT_OK : fail(h, MOT_ENOCONV, "GMRES reached its iteration limit");
}

// x solves Q_0 x = rhs by right-preconditioned GMRES: Q_0 M z = rhs, x = M z,
// with M the FP32 copy of Q_0^{-1} (mixed path) or its FP64 form (FP64 path
// with fp64_precond). z lives in a buffer that apply_q0 does not touch: W.pd
// on the mixed path (dense Q_0), W.s1 on the FP64 path (its product-form Q_0
// uses W.pd inside the left factor; the history sums in W.s1 are consumed
// before the solve). rhs must not be W.r, W.q1 or that buffer.
int prec_solve(mot_handle* h, const Work& W, const double* rhs, double* x, double tol, cudaStream_t s) {
    double* z = mixed(h) ? W.pd : W.s1;
    h->prec_active = true;
    int st = gmres(h, W, rhs, z, false, tol, s);
    h->prec_active = false;
    if (!mixed(h)) {
        launch_gemm_rect(h, 2 * h->npad, 2 * h->npad, h->d_Minv64, z, h->B, x, s);
    } else if (h->emu_Minv.a16) {
        launch_emu_gemm(h, h->emu_Minv, W.pd, h->B, x, s);
    } else {
        launch_d2f(h, (size_t)h->npad * 2 * h->B, W.pd, h->d_xf, s);
        launch_sgemm_d(h, 2 * h->npad, h->B, 2 * h->npad, h->d_Minvf, h->d_xf, x, s);
    }
    return st;
}

int ensure_state(mot_handle* h, int B) {
    if (h->B == B && h->d_ring) return MOT_OK;
    if (h->B != 0 && h->B != B) return fail(h, MOT_EINVAL, "batch size changed without mot_reset");
    h->B = B;
    const size_t bv = (size_t)h->npad * 2 * B;
    h->gm_m = std::min(std::max(h->opt.gmres_maxit, 1), 100);
    h->d_waves = (double*)dalloc(h, sizeof(double) * 10 * B);
    h->d_ring = (double*)dalloc(h, sizeof(double) * (size_t)h->R * 6 * bv);
    h->d_win = (double*)dalloc(h, sizeof(double) * (size_t)(h->max_tail_lag + 1) * bv);
    h->d_cur = (double*)dalloc(h, sizeof(double) * 4 * (size_t)h->npad * B);
    if (h->opt.precision == MOT_PREC_MIXED && !h->precomputing) {
        int major = 0;
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, h->dev);
        h->hist_tc = mflag(h, MOT_MIX_HIST32) && mflag(h, MOT_MIX_TC) && B % 8 == 0 && major == 10 &&
                      history_tc_fits(h->npad, h->tc_bulk) && h->hist_tc_list.packed;
        if (h->hist_tc && !h->d_tiles16) {  // operator data: kept until mot_destroy
            // ntiles + 1 tiles: the last one stays zero (the missing partner of a merged task)
            h->d_tiles16 =
                (uint16_t*)dalloc(h, sizeof(uint16_t) * 3 * (size_t)(h->ntiles + 1) * MOT_TILE * MOT_TILE);
            if (!h->d_tiles16) return fail(h, MOT_EOOM, "device allocation (tensor-core tiles)");
            launch_split_tiles(h, 0);
            CK(cudaDeviceSynchronize());
        }
        if (h->hist_tc) {
            h->d_ring16 = (uint16_t*)dalloc(h, sizeof(uint16_t) * (size_t)h->R * history_tc_ring_slot_elems(h));
            h->d_win16 = (uint16_t*)dalloc(h, sizeof(uint16_t) * (size_t)(h->max_tail_lag + 1) *
                                                  history_tc_ring_slot_elems(h) / 2);
            if (!h->d_ring16 || !h->d_win16) return fail(h, MOT_EOOM, "device allocation of the march state");
        } else {
            h->d_ring32 = (float*)dalloc(h, sizeof(float) * (size_t)h->R * 6 * bv);
            h->d_win32 = (float*)dalloc(h, sizeof(float) * (size_t)(h->max_tail_lag + 1) * bv);
            if (!h->d_ring32 || !h->d_win32) return fail(h, MOT_EOOM, "device allocation of the march state");
        }
        h->d_xf = (float*)dalloc(h, sizeof(float) * 2 * bv);
        if (!h->d_xf) return fail(h, MOT_EOOM, "device allocation of the march state");
        if (h->d_Lfinvf) {
            const size_t blk = (size_t)h->nfpd * 2 * B;
            h->d_pcg_work = (double*)dalloc(h, sizeof(double) * (4 * blk + (size_t)((h->nfpd + 63) / 64) * 2 * B));
            h->d_pcg_scal = (double*)dalloc(h, sizeof(double) * 8 * 2 * B);
            h->d_pcg_f32 = (float*)dalloc(h, sizeof(float) * blk);
            if (!h->d_pcg_work || !h->d_pcg_scal || !h->d_pcg_f32)
                return fail(h, MOT_EOOM, "device allocation of the march state");
        }
    }
    h->d_wprev1 = (double*)dalloc(h, sizeof(double) * bv);
    h->d_wprev2 = (double*)dalloc(h, sizeof(double) * bv);
    if (!h->d_wprev1 || !h->d_wprev2) return fail(h, MOT_EOOM, "device allocation of the march state");
    h->d_dft = (double*)dalloc(h, sizeof(double) * std::max(1, h->nfreq) * 4 * (size_t)h->npad * B * 2);
    h->work_bytes = sizeof(double) * work_doubles(h);
    h->d_work = (double*)dalloc(h, h->work_bytes);
    int maxch = std::max(std::max(h->hist.nchunks, h->lag0.nchunks), h->hist_tc_list.nchunks);
    h->partial_bytes = sizeof(double) * (size_t)std::max(1, maxch) * 2 * MOT_TILE * 2 * B;
    h->d_partial = (double*)dalloc(h, h->partial_bytes);
    h->d_V = (double*)dalloc(h, sizeof(double) * (size_t)(h->gm_m + 1) * bv);
    h->d_H = (double*)dalloc(h, sizeof(double) * (size_t)B * (h->gm_m + 1) * h->gm_m);
    h->d_g = (double*)dalloc(h, sizeof(double) * (size_t)B * (h->gm_m + 1));
    h->d_cs = (double*)dalloc(h, sizeof(double) * (size_t)B * h->gm_m);
    h->d_sn = (double*)dalloc(h, sizeof(double) * (size_t)B * h->gm_m);
    h->red_bytes = sizeof(double) * (size_t)((h->npad + 255) / 256 + 1) * (h->gm_m + 1) * B;
    h->d_red = (double*)dalloc(h, h->red_bytes);
    h->d_resid = (double*)dalloc(h, sizeof(double) * B);
    h->d_gm_active = (int*)dalloc(h, sizeof(int) * B);
    h->d_gm_jend = (int*)dalloc(h, sizeof(int) * B);
    h->d_gm_bnorm = (double*)dalloc(h, sizeof(double) * B);
    h->d_wscale = (double*)dalloc(h, sizeof(double) * B);
    if (!h->d_waves || !h->d_ring || !h->d_win || !h->d_cur || !h->d_dft || !h->d_work || !h->d_partial ||
        !h->d_V || !h->d_H || !h->d_g || !h->d_cs || !h->d_sn || !h->d_red || !h->d_resid || !h->d_gm_active ||
        !h->d_gm_jend || !h->d_gm_bnorm || !h->d_wscale)
        return fail(h, MOT_EOOM, "device allocation of the march state");
    h->h_waves.assign(10 * B, NAN);
    return MOT_OK;
}

void free_state(mot_handle* h) {
    void* ptrs[] = {h->d_waves, h->d_ring, h->d_win, h->d_cur, h->d_dft, h->d_work, h->d_partial, h->d_V, h->d_H,
                    h->d_g, h->d_cs, h->d_sn, h->d_red, h->d_resid, h->d_gm_active, h->d_gm_jend, h->d_gm_bnorm,
                    h->d_wscale,
                    h->d_wprev1, h->d_wprev2};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    h->d_wprev1 = h->d_wprev2 = nullptr;
    void* fptrs[] = {h->d_ring32, h->d_win32, h->d_xf, h->d_pcg_work, h->d_pcg_scal, h->d_pcg_f32, h->d_ring16,
                     h->d_win16};
    for (void* p : fptrs)
        if (p) cudaFree(p);
    h->d_ring32 = h->d_win32 = h->d_xf = h->d_pcg_f32 = nullptr;
    h->d_ring16 = h->d_win16 = nullptr;
    h->hist_tc = false;
    h->d_pcg_work = h->d_pcg_scal = nullptr;
    h->d_waves = h->d_ring = h->d_win = h->d_cur = h->d_dft = h->d_work = h->d_partial = nullptr;
    h->d_V = h->d_H = h->d_g = h->d_cs = h->d_sn = h->d_red = h->d_resid = nullptr;
    h->d_gm_active = h->d_gm_jend = nullptr;
    h->d_gm_bnorm = nullptr;
    h->d_wscale = nullptr;
    h->B = 0;
    h->step = 0;
    h->gmres_iters_total = 0;
}

int check_waves(mot_handle* h, const mot_wave* waves, int B) {
    for (int b = 0; b < B; b++) {
        const mot_wave& w = waves[b];
        double v[10] = {w.A, w.p[0], w.p[1], w.p[2], w.k[0], w.k[1], w.k[2], w.w, w.t0, w.t_trunc};
        for (double x : v)
            if (!std::isfinite(x)) return fail(h, MOT_EINVAL, "non-finite plane-wave parameter");
        if (!(w.w > 0)) return fail(h, MOT_EINVAL, "plane-wave width must be > 0");
    }
    return MOT_OK;
}

int upload_waves(mot_handle* h, const mot_wave* waves, int B, cudaStream_t s) {
    std::vector<double> v(10 * B);
    for (int b = 0; b < B; b++) {
        const mot_wave& w = waves[b];
        double t[10] = {w.A, w.p[0], w.p[1], w.p[2], w.k[0], w.k[1], w.k[2], w.w, w.t0, w.t_trunc};
        memcpy(&v[10 * b], t, sizeof t);
    }
    // the step's input is copied every step (B x 80 bytes)
    h->h_waves = v;
    CK(cudaMemcpyAsync(h->d_waves, h->h_waves.data(), sizeof(double) * 10 * B, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    return MOT_OK;
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// One MOT step in three phases (a full step runs all of them on one stream):
//   STEP_INPUTS   right-hand side, windowed sums of the K~ tail, reduced-precision panels
//   STEP_HISTORY  the history contraction into W.s1, W.s2
//   STEP_SOLVE    combine, left factor, Q_0 solve, ring update, recovery
// mot_run_many runs the history of several scatterers as one launch between
// their STEP_INPUTS and STEP_SOLVE phases.
enum { STEP_INPUTS = 1, STEP_HISTORY = 2, STEP_SOLVE = 4, STEP_ALL = 7 };

int do_step(mot_handle* h, cudaStream_t s, int phases = STEP_ALL) {
    Work W = work_of(h);
    const long long i = h->step + 1;
    const int n = h->npad * 2 * h->B;
    const size_t bv = (size_t)n;
#define PEV(k) \
    if (h->pev[0]) cudaEventRecord(h->pev[k], s)
    const bool mx = mixed(h);
    const bool h32 = mx && mflag(h, MOT_MIX_HIST32);
    if (phases & STEP_INPUTS) {
        CK(cudaMemsetAsync(h->d_cg_iters, 0, 3 * sizeof(int), s));
        PEV(0);
        launch_rhs(h, i, W.rho1, W.rho2, s);
        PEV(1);
        if (i >= 2) {
            launch_window_sums(h, i, s);
            if (h->hist_tc) {
                if (h->max_tail_lag >= 1) launch_split3(h, h->max_tail_lag + 1, h->d_win, h->d_win16, s);
            } else if (h32) {
                if (h->max_tail_lag >= 1)
                    launch_d2f(h, (size_t)(h->max_tail_lag + 1) * bv, h->d_win, h->d_win32, s);
            }
        }
    }
    if ((phases & STEP_HISTORY) && i >= 2) {
        if (h->hist_tc && !(h->hist_tc_list.packed && h->hist_tc_list.rb_ptr && h->hist_tc_list.rb_chunks))
            return fail(h, MOT_ESTATE, "tensor-core history: no task list (a re-cut of the list failed)");
        if (h->hist_tc)
            launch_history_tc(h, h->hist_tc_list, i, W.s1, W.s2, s);
        else if (h32)
            launch_history32(h, h->hist, h->d_tiles32, h->d_ring32, h->d_win32, nullptr, 0, i, W.s1, W.s2, s);
        else
            launch_history(h, h->hist, h->d_tiles, h->d_ring, h->d_win, nullptr, 0, i, W.s1, W.s2, s);
    }
    if (!(phases & STEP_SOLVE)) return MOT_OK;
    if (i >= 2) {
        launch_axpby(h, n, 1.0, W.rho1, -1.0, W.s1, W.y1, s);
        launch_axpby(h, n, 1.0, W.rho2, -1.0, W.s2, W.y2, s);
    } else {
        launch_axpby(h, n, 1.0, W.rho1, 0.0, nullptr, W.y1, s);
        launch_axpby(h, n, 1.0, W.rho2, 0.0, nullptr, W.y2, s);
    }
    PEV(2);
    if (mx) {
        // b = [M1 | M2] [y1; y2] (y1, y2 are adjacent block vectors)
        if (mflag(h, MOT_MIX_LF32)) {
            launch_d2f(h, 2 * bv, W.y1, h->d_xf, s);
            launch_sgemm_d(h, h->npad, 2 * h->B, 2 * h->npad, h->d_LFf, h->d_xf, W.b, s);
        } else {
            if (h->emu_LF.a16)  // emulated FP64 on the tensor cores (MOT_MIX_EMU64)
                launch_emu_gemm(h, h->emu_LF, W.y1, 2 * h->B, W.b, s);
            else
                launch_gemm_rect(h, h->npad, 2 * h->npad, h->d_LF, W.y1, 2 * h->B, W.b, s);
        }
    } else {
        left_factor(h, W, W.y1, W.y2, W.b, s);
    }
    PEV(3);
    // initial guess: linear extrapolation of the last two solutions
    bool have_x0 = i >= 2;
    if (i >= 3)
        launch_axpby(h, n, 2.0, h->d_wprev1, -1.0, h->d_wprev2, W.x, s);
    else if (i == 2)
        launch_axpby(h, n, 1.0, h->d_wprev1, 0.0, nullptr, W.x, s);
    // every wave's system is solved at O(1) magnitude: b and the initial
    // guess scaled by a power of two (exact), the solution scaled back. Late
    // in a march the solution decays without bound; unscaled, the sums of
    // squares of the solve (and the FP32 copies of the mixed path) would
    // underflow long before the values themselves do.
    launch_wave_scale(h, W.b, h->d_wscale, s);
    launch_wave_apply(h, h->d_wscale, false, W.b, s);
    if (have_x0) launch_wave_apply(h, h->d_wscale, false, W.x, s);
    const bool refine = mx && mflag(h, MOT_MIX_REFINE);
    const bool prec = (mx && h->d_Minvf) || (!mx && h->d_Minv64);
    // with refinement the reduced-precision solves only need 1e-6: each sweep gains ~6 digits
    const double tol_in = refine ? std::max(h->opt.gmres_tol, 1e-6) : h->opt.gmres_tol;
    int st = prec ? prec_solve(h, W, W.b, W.x, tol_in, s) : gmres(h, W, W.b, W.x, have_x0, tol_in, s);
    if (st != MOT_OK && st != MOT_ENOCONV) return st;
    PEV(4);
    h->refine_sweeps = 0;
    if (refine) {
        // FP64 iterative refinement: r = b - Q_0 x with the FP64 dense Q_0,
        // correction from the reduced-precision GMRES, until |r| <= gmres_tol |b|
        const int gm_iters = h->last_gmres_iters;
        // default: one FP64 residual and one correction (no residual re-check after it)
        const int max_sweeps = h->opt.refine_sweeps > 0 ? h->opt.refine_sweeps : 1;
        for (int sweep = 0; sweep < max_sweeps; sweep++) {
            apply_q0_dense64(h, W.x, W.r, s);
            launch_axpby(h, n, 1.0, W.b, -1.0, W.r, W.r, s);
            launch_gm_norm(h, W.r, W.nrm, s);
            launch_gm_norm(h, W.b, W.beta, s);
            std::vector<double> rn(h->B), bn(h->B);
            CK(cudaMemcpyAsync(rn.data(), W.nrm, sizeof(double) * h->B, cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(bn.data(), W.beta, sizeof(double) * h->B, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            double worst = 0;
            for (int b = 0; b < h->B; b++) worst = std::max(worst, bn[b] > 0 ? rn[b] / bn[b] : 0.0);
            h->last_gmres_resid = worst;
            if (worst <= h->opt.gmres_tol) break;
            h->refine_sweeps++;
            // W.tmp receives the correction d of Q_0 d = r (r copied to W.dd: gmres uses W.r)
            launch_axpby(h, n, 1.0, W.r, 0.0, nullptr, W.dd, s);
            int st2 = prec ? prec_solve(h, W, W.dd, W.tmp, 1e-6, s) : gmres(h, W, W.dd, W.tmp, false, 1e-6, s);
            if (st2 != MOT_OK && st2 != MOT_ENOCONV) return st2;
            launch_axpby(h, n, 1.0, W.x, 1.0, W.tmp, W.x, s);
        }
        h->last_gmres_iters = gm_iters;
    }
    launch_wave_apply(h, h->d_wscale, true, W.x, s);
    PEV(5);
    h->gmres_iters_total += h->last_gmres_iters;
    std::swap(h->d_wprev1, h->d_wprev2);
    CK(cudaMemcpyAsync(h->d_wprev1, W.x, sizeof(double) * bv, cudaMemcpyDeviceToDevice, s));
    // ring slot i: variants of l_i and s_i
    project_sigma(h, W, W.x, W.sig, s);
    launch_axpby(h, n, 1.0, W.x, -1.0, W.sig, W.ell, s);
    const int slot = (int)(i % h->R);
    launch_variants(h, W.ell, h->d_ring + ((size_t)slot * 2 + 0) * 3 * bv, h->eta, h->etap, s);
    launch_variants(h, W.sig, h->d_ring + ((size_t)slot * 2 + 1) * 3 * bv, h->eta, h->etap, s);
    if (h->hist_tc)
        launch_split_ring(h, slot, s);
    else if (mx)
        launch_d2f(h, 6 * bv, h->d_ring + (size_t)slot * 6 * bv, h->d_ring32 + (size_t)slot * 6 * bv, s);
    PEV(6);
    h->step = i;
    launch_recover(h, i, s);
    PEV(7);
#undef PEV
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h->h_cg_iters, h->d_cg_iters, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h->pev[0]) {
        for (int k = 0; k < 7; k++) {
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, h->pev[k], h->pev[k + 1]));
            h->phase_ms[k] += ms;
        }
    }
    if (h->ev_pending) {
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
        h->timed_ms += ms;
        h->timed_launches++;
        h->ev_pending = false;
    }
    h->last_cg_iters = h->h_cg_iters[0];
    if (h->h_cg_iters[2] != 0)
        return fail(h, MOT_ECUDA,
                    "tensor-core history: a pipeline wait ran out of time (code " + std::to_string(h->h_cg_iters[2]) +
                        ")");
    if (h->h_cg_iters[1] > 0) return fail(h, MOT_ENOCONV, "a projector or Gram CG solve reached its iteration limit");
    return st;
}

}  // namespace

// ============================================================== C ABI

MOT_API int mot_create(const mot_mesh* mesh, double eps_r, double mu_r, double dt, int K, const mot_options* opt,
                       mot_handle** out) {
    if (!out) return MOT_EINVAL;
    *out = nullptr;
    mot_handle* h = new mot_handle();
    h->opt.precision = MOT_PREC_FP64;
    h->opt.device = 0;
    h->opt.gmres_tol = 1e-13;
    h->opt.gmres_maxit = 200;
    h->opt.cg_tol = 1e-14;
    h->opt.cg_maxit = 5000;
    if (opt) {
        h->opt.precision = opt->precision;
        h->opt.device = opt->device;
        if (opt->gmres_tol > 0) h->opt.gmres_tol = opt->gmres_tol;
        if (opt->gmres_maxit > 0) h->opt.gmres_maxit = opt->gmres_maxit;
        if (opt->cg_tol > 0) h->opt.cg_tol = opt->cg_tol;
        if (opt->cg_maxit > 0) h->opt.cg_maxit = opt->cg_maxit;
        h->opt.timing = opt->timing;
        h->opt.mixed_flags = opt->mixed_flags;
        h->opt.refine_sweeps = opt->refine_sweeps;
        h->opt.fp64_precond = opt->fp64_precond;
        h->opt.hist_stall_test = opt->hist_stall_test;
        h->opt.fp64_direct = opt->fp64_direct;
    }
    auto bad = [&](const char* m) {
        h->err = m;
        *out = h;  // keep the handle so the caller can read the message
        return MOT_EINVAL;
    };
    if (!mesh || !mesh->verts || !mesh->tris || mesh->nv < 4 || mesh->nf < 4) return bad("mesh missing or too small");
    if (!(eps_r > 0) || !(mu_r > 0) || !(dt > 0) || !std::isfinite(eps_r) || !std::isfinite(mu_r) || !std::isfinite(dt))
        return bad("eps_r, mu_r and dt must be finite and > 0");
    if (h->opt.precision != MOT_PREC_FP64 && h->opt.precision != MOT_PREC_MIXED) return bad("unknown precision");
    if (h->opt.precision == MOT_PREC_MIXED && !(opt && opt->gmres_tol > 0)) h->opt.gmres_tol = 1e-11;
    if (h->opt.mixed_flags == 0) h->opt.mixed_flags = MOT_MIX_DEFAULT;
    h->nv = mesh->nv;
    h->nf = mesh->nf;
    h->verts.assign(mesh->verts, mesh->verts + 3 * (size_t)h->nv);
    h->tris.assign(mesh->tris, mesh->tris + 3 * (size_t)h->nf);
    for (double v : h->verts)
        if (!std::isfinite(v)) return bad("non-finite vertex coordinate");
    for (int t : h->tris)
        if (t < 0 || t >= h->nv) return bad("triangle vertex index out of range");
    // canonical edges: directed a->b of every face; the face is c+ of (a,b) if a < b
    std::map<std::pair<int, int>, std::pair<int, int>> dir;  // (a,b) -> (face, opposite)
    for (int f = 0; f < h->nf; f++) {
        const int* t = &h->tris[3 * f];
        for (int j = 0; j < 3; j++) {
            int a = t[j], b = t[(j + 1) % 3], o = t[(j + 2) % 3];
            if (a == b) return bad("degenerate triangle");
            if (!dir.emplace(std::make_pair(a, b), std::make_pair(f, o)).second)
                return bad("repeated directed edge: mesh is non-manifold or inconsistently oriented");
        }
    }
    for (auto& kv : dir) {
        int a = kv.first.first, b = kv.first.second;
        auto it = dir.find({b, a});
        if (it == dir.end()) return bad("open or inconsistently oriented mesh");
        if (a < b) {
            h->ev.push_back(a);
            h->ev.push_back(b);
            h->ef.push_back(kv.second.first);
            h->ef.push_back(it->second.first);
            h->eo.push_back(kv.second.second);
            h->eo.push_back(it->second.second);
        }
    }
    h->ne = (int)h->ev.size() / 2;
    if (2 * h->ne != 3 * h->nf) return bad("edge count is not 3F/2");
    // material, D, T_max, k_max (Eq. (alpha), Section V-B)
    h->eps_r = eps_r;
    h->mu_r = mu_r;
    h->dt = dt;
    h->c = 1.0;
    h->eta = 1.0;
    h->cp = 1.0 / sqrt(eps_r * mu_r);
    h->etap = sqrt(mu_r / eps_r);
    double D2 = 0;
    for (int a = 0; a < h->nv; a++)
        for (int b = a + 1; b < h->nv; b++) {
            double d0 = h->verts[3 * a] - h->verts[3 * b], d1 = h->verts[3 * a + 1] - h->verts[3 * b + 1],
                   d2 = h->verts[3 * a + 2] - h->verts[3 * b + 2];
            D2 = std::max(D2, d0 * d0 + d1 * d1 + d2 * d2);
        }
    h->D = sqrt(D2);
    h->tmax = h->D / std::min(h->c, h->cp);
    double r = h->tmax / dt;
    double rn = std::round(r);
    h->kmax = (fabs(r - rn) < 1e-12 * std::max(1.0, r)) ? (int)rn : (int)ceil(r);
    if (K < h->kmax + 1) {
        char buf[160];
        snprintf(buf, sizeof buf, "K = %d is smaller than k_max + 1 = %d", K, h->kmax + 1);
        return bad(buf);
    }
    h->K = h->kmax + 1;
    h->R = h->K + 1;
    // Morton order of the edge midpoints (internal row order)
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int v = 0; v < h->nv; v++)
        for (int d = 0; d < 3; d++) {
            lo[d] = std::min(lo[d], h->verts[3 * v + d]);
            hi[d] = std::max(hi[d], h->verts[3 * v + d]);
        }
    std::vector<std::pair<uint64_t, int>> keys(h->ne);
    for (int e = 0; e < h->ne; e++) {
        uint64_t code = 0;
        for (int d = 0; d < 3; d++) {
            double m = 0.5 * (h->verts[3 * h->ev[2 * e] + d] + h->verts[3 * h->ev[2 * e + 1] + d]);
            double u = (hi[d] > lo[d]) ? (m - lo[d]) / (hi[d] - lo[d]) : 0.0;
            uint64_t q = (uint64_t)std::min(2097151.0, std::max(0.0, u * 2097151.0));
            code |= spread3(q) << d;
        }
        keys[e] = {code, e};
    }
    std::sort(keys.begin(), keys.end());
    h->perm.resize(h->ne);
    h->iperm.resize(h->ne);
    for (int p = 0; p < h->ne; p++) {
        h->perm[p] = keys[p].second;
        h->iperm[keys[p].second] = p;
    }
    h->npad = (h->ne + MOT_TILE - 1) / MOT_TILE * MOT_TILE;
    h->nrb = h->npad / MOT_TILE;
    // device
    cudaError_t ce = cudaSetDevice(h->opt.device);
    if (ce != cudaSuccess) {
        *out = h;
        return cuda_fail(h, ce, "cudaSetDevice");
    }
    h->dev = h->opt.device;
    // incidence on the internal order
    std::vector<int> efi(2 * h->ne), evi(2 * h->ne);
    for (int p = 0; p < h->ne; p++) {
        int e = h->perm[p];
        efi[2 * p] = h->ef[2 * e];
        efi[2 * p + 1] = h->ef[2 * e + 1];
        evi[2 * p] = h->ev[2 * e];
        evi[2 * p + 1] = h->ev[2 * e + 1];
    }
    std::vector<int> fe(3 * h->nf, -1);
    std::vector<double> fs(3 * h->nf, 0.0);
    std::vector<int> fill(h->nf, 0);
    std::vector<std::tuple<int, int, double>> tv, tlf, tlv;
    for (int p = 0; p < h->ne; p++) {
        for (int side = 0; side < 2; side++) {
            int f = efi[2 * p + side];
            int k = fill[f]++;
            if (k >= 3) return bad("face with more than three edges");
            fe[3 * f + k] = p;
            fs[3 * f + k] = side == 0 ? 1.0 : -1.0;
        }
        tv.emplace_back(evi[2 * p + 1], p, 1.0);
        tv.emplace_back(evi[2 * p], p, -1.0);
        int fp = efi[2 * p], fm = efi[2 * p + 1];
        tlf.emplace_back(fp, fp, 1.0);
        tlf.emplace_back(fm, fm, 1.0);
        tlf.emplace_back(fp, fm, -1.0);
        tlf.emplace_back(fm, fp, -1.0);
        int vm = evi[2 * p], vp = evi[2 * p + 1];
        tlv.emplace_back(vp, vp, 1.0);
        tlv.emplace_back(vm, vm, 1.0);
        tlv.emplace_back(vp, vm, -1.0);
        tlv.emplace_back(vm, vp, -1.0);
    }
    HostCsr VE = csr_from_triplets(h->nv, h->ne, tv);
    HostCsr LF = csr_from_triplets(h->nf, h->nf, tlf);
    HostCsr LV = csr_from_triplets(h->nv, h->nv, tlv);
    h->d_edge_faces = (int*)dalloc(h, sizeof(int) * 2 * h->ne);
    h->d_edge_verts = (int*)dalloc(h, sizeof(int) * 2 * h->ne);
    h->d_face_edges = (int*)dalloc(h, sizeof(int) * 3 * h->nf);
    h->d_face_sgn = (double*)dalloc(h, sizeof(double) * 3 * h->nf);
    h->d_iperm = (int*)dalloc(h, sizeof(int) * h->ne);
    h->d_cg_iters = (int*)dalloc(h, sizeof(int) * 4);
    *out = h;
    if (!h->d_edge_faces || !h->d_edge_verts || !h->d_face_edges || !h->d_face_sgn || !h->d_iperm || !h->d_cg_iters)
        return fail(h, MOT_EOOM, "device allocation (topology)");
    CK(cudaMemcpy(h->d_edge_faces, efi.data(), sizeof(int) * 2 * h->ne, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_edge_verts, evi.data(), sizeof(int) * 2 * h->ne, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_face_edges, fe.data(), sizeof(int) * 3 * h->nf, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_face_sgn, fs.data(), sizeof(double) * 3 * h->nf, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_iperm, h->iperm.data(), sizeof(int) * h->ne, cudaMemcpyHostToDevice));
    CK(cudaMallocHost(&h->h_cg_iters, sizeof(int) * 4));
    CK(cudaEventCreateWithFlags(&h->ev_state, cudaEventDisableTiming));
    if (h->opt.timing) {
        CK(cudaEventCreate(&h->ev0));
        CK(cudaEventCreate(&h->ev1));
        for (int k = 0; k < 8; k++) CK(cudaEventCreate(&h->pev[k]));
    }
    int st;
    if ((st = upload_csr(h, VE, h->vtx_edges)) != MOT_OK) return st;
    if ((st = upload_csr(h, LF, h->Lf)) != MOT_OK) return st;
    if ((st = upload_csr(h, LV, h->Lv)) != MOT_OK) return st;
    return MOT_OK;
}

namespace {

// tile kinds: 0 A.T ext, 1 A.T int, 2 A.K (ext+int), 3 Ah.T ext, 4 Ah.T int, 5 Ah.K, 6 At.T ext, 7 At.T int,
// 8 At.K explicit, 9 At.K tails (window slices)
constexpr int NTK = 10;
const int kMatKind[12] = {0, 2, 3, 5, 6, 8, 1, 2, 4, 5, 7, 8};
const int kKindVariant[NTK] = {0, 1, 2, 0, 1, 2, 0, 1, 2, 2};
const int kKindFamily[NTK] = {0, 0, 0, 1, 1, 1, 2, 2, 2, 3};  // 0 A, 1 Ah, 2 At, 3 tail

// Task list of the tensor-core history kernel. Every coefficient panel
// (part, variant, lag, column block) of a row block multiplies at most one
// tile per output (A_k and A~_k on l, A_k and A^_k on s): the two are merged
// into one task that gathers the panel once and multiplies both tiles, the
// missing one replaced by a zero tile. To keep the rows of the lags in use
// resident in L2, the list is cut into (lag range, row block) pieces ordered
// lag range first, so the CTAs that run at the same time work on the same few
// lags. Within a piece: coefficient transform (variant; windowed sums
// separately), lag, column block.
// cap: most tasks per chunk; lag_frac: the fraction of the L2 that the ring
// slots of one lag range may fill (sets the lags per range).
int make_tc_list(mot_handle* h, const std::vector<HistTask>& tasks, const std::vector<int>& rbs, int cap,
                 double lag_frac) {
    const int nrb = h->nrb;
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, h->dev);
    if (l2 <= 0) l2 = 64 << 20;
    // bf16 slices of l and s of one lag for B = 64: 2 parts x 3 slices x npad x 128 x 2 bytes
    const double lag_bytes = 2.0 * 3.0 * h->npad * 128.0 * 2.0;
    const int kr = std::max(1, (int)(lag_frac * l2 / lag_bytes));
    {  // a list made before (re-tuning) is replaced
        TaskList& old = h->hist_tc_list;
        void* ptrs[] = {old.packed, old.chunks, old.rb_ptr, old.rb_chunks};
        for (void* p : ptrs)
            if (p) cudaFree(p);
        old.packed = nullptr;
        old.chunks = nullptr;
        old.rb_ptr = old.rb_chunks = nullptr;
        old.ntasks = old.nchunks = old.cap = 0;
    }
    auto xform = [](int code) { return (code & 3) == 2 ? 3 : (code >> 2) & 3; };
    const unsigned zt = (unsigned)h->ntiles;  // index of the zero tile
    struct Merged {
        int rb, cb, k, code;  // code = part | variant << 2
        unsigned tile[2];
    };
    std::vector<size_t> ord(tasks.size());
    std::iota(ord.begin(), ord.end(), (size_t)0);
    auto mkey = [&](size_t t) {
        return std::make_tuple(rbs[t], tasks[t].cb, tasks[t].k, tasks[t].code & 15);
    };
    std::sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return mkey(a) < mkey(b); });
    std::vector<Merged> m;
    m.reserve(tasks.size() / 2 + 16);
    for (size_t q = 0; q < ord.size(); q++) {
        const size_t t = ord[q];
        const HistTask& x = tasks[t];
        const int out = (x.code >> 4) & 1;
        if (q == 0 || mkey(t) != mkey(ord[q - 1])) m.push_back(Merged{rbs[t], x.cb, x.k, x.code & 15, {zt, zt}});
        if (m.back().tile[out] != zt) return MOT_OK;  // two tiles for one output and panel: no tensor path
        m.back().tile[out] = (unsigned)x.tile;
    }
    std::sort(m.begin(), m.end(), [&](const Merged& a, const Merged& b) {
        const int ra = (a.k - 1) / kr, rbb = (b.k - 1) / kr;
        if (ra != rbb) return ra < rbb;
        if (a.rb != b.rb) return a.rb < b.rb;
        if (xform(a.code) != xform(b.code)) return xform(a.code) < xform(b.code);
        if (a.k != b.k) return a.k < b.k;
        return a.cb < b.cb;
    });
    cap = std::max(1, std::min(cap, MOT_TC_CHUNK));  // tasks per chunk (staged in the CTA's shared memory)
    int maxcount = 0;
    std::vector<HistChunk> chunks;
    std::vector<std::vector<int>> per_rb(nrb);
    size_t i = 0;
    while (i < m.size()) {
        const int rb = m[i].rb, r = (m[i].k - 1) / kr;
        size_t j = i;
        while (j < m.size() && m[j].rb == rb && (m[j].k - 1) / kr == r && (int)(j - i) < cap) j++;
        per_rb[rb].push_back((int)chunks.size());
        chunks.push_back(HistChunk{rb, (int)i, (int)(j - i)});
        maxcount = std::max(maxcount, (int)(j - i));
        i = j;
    }
    std::vector<int> rptr(nrb + 1, 0), rch;
    for (int rb = 0; rb < nrb; rb++) {
        rptr[rb] = (int)rch.size();
        rch.insert(rch.end(), per_rb[rb].begin(), per_rb[rb].end());
    }
    rptr[nrb] = (int)rch.size();
    std::vector<uint4> packed(m.size());
    for (size_t t = 0; t < m.size(); t++) {
        const Merged& x = m[t];
        if (x.cb > 0xFFFF || x.k > 0x3FF) return MOT_OK;  // outside the packed range: no tensor path
        packed[t] = make_uint4(x.tile[0], x.tile[1], (unsigned)x.cb | ((unsigned)x.k << 16) | ((unsigned)x.code << 26), 0u);
    }
    TaskList& tl = h->hist_tc_list;
    tl.ntasks = (int)m.size();
    tl.nchunks = (int)chunks.size();
    tl.cap = std::max(1, maxcount);
    h->tc_cap = cap;
    h->tc_lag_frac = lag_frac;
    tl.packed = (uint4*)dalloc(h, sizeof(uint4) * std::max<size_t>(1, packed.size()));
    tl.chunks = (HistChunk*)dalloc(h, sizeof(HistChunk) * std::max<size_t>(1, chunks.size()));
    tl.rb_ptr = (int*)dalloc(h, sizeof(int) * (nrb + 1));
    tl.rb_chunks = (int*)dalloc(h, sizeof(int) * std::max<size_t>(1, rch.size()));
    if (!tl.packed || !tl.chunks || !tl.rb_ptr || !tl.rb_chunks)
        return fail(h, MOT_EOOM, "device allocation (tensor-core task list)");
    if (!packed.empty()) CK(cudaMemcpy(tl.packed, packed.data(), sizeof(uint4) * packed.size(), cudaMemcpyHostToDevice));
    if (!chunks.empty()) CK(cudaMemcpy(tl.chunks, chunks.data(), sizeof(HistChunk) * chunks.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(tl.rb_ptr, rptr.data(), sizeof(int) * (nrb + 1), cudaMemcpyHostToDevice));
    if (!rch.empty()) CK(cudaMemcpy(tl.rb_chunks, rch.data(), sizeof(int) * rch.size(), cudaMemcpyHostToDevice));
    return MOT_OK;
}

int build_tiles(mot_handle* h, const mot_operators* ops) {
    const int T = MOT_TILE;
    const int nrb = h->nrb;
    const int L = h->kmax + 2;  // lags 0 .. kmax+1
    std::vector<int> id((size_t)NTK * L * nrb * nrb, -1);
    auto key = [&](int kind, int k, int rb, int cb) { return (((size_t)kind * L + k) * nrb + rb) * nrb + cb; };
    // Column order of every row block: all edges sorted by the distance of their
    // midpoint from the block's centroid. Interactions are shell shaped (lag k
    // couples edges about k c dt apart), so columns at similar distance share
    // their nonzero lags and the (row block x 32 sorted columns) tiles are dense.
    const int np = h->npad;
    std::vector<double> mid(3 * (size_t)h->ne);
    for (int p = 0; p < h->ne; p++) {
        const int e = h->perm[p];
        for (int d = 0; d < 3; d++)
            mid[3 * p + d] = 0.5 * (h->verts[3 * h->ev[2 * e] + d] + h->verts[3 * h->ev[2 * e + 1] + d]);
    }
    std::vector<int> colidx((size_t)nrb * np, h->ne < np ? h->ne : 0), colpos((size_t)nrb * np, 0);
    if (h->tc_bulk) {
        // bulk form of the tensor-core history: one global column order (the
        // Morton order of the rows), so that the coefficient panel of column
        // block cb is the contiguous ring rows [32 cb, 32 cb + 32)
        for (int rb = 0; rb < nrb; rb++)
            for (int j = 0; j < np; j++) {
                colidx[(size_t)rb * np + j] = j;
                colpos[(size_t)rb * np + j] = j;
            }
    } else {
        auto sort_rb = [&](int t0, int nth) {
            std::vector<std::pair<double, int>> dist(h->ne);
            for (int rb = t0; rb < nrb; rb += nth) {
                double c[3] = {0, 0, 0};
                int cnt = 0;
                for (int p = rb * T; p < std::min(h->ne, rb * T + T); p++, cnt++)
                    for (int d = 0; d < 3; d++) c[d] += mid[3 * p + d];
                for (int d = 0; d < 3; d++) c[d] /= std::max(1, cnt);
                for (int p = 0; p < h->ne; p++) {
                    double dx = mid[3 * p] - c[0], dy = mid[3 * p + 1] - c[1], dz = mid[3 * p + 2] - c[2];
                    dist[p] = {dx * dx + dy * dy + dz * dz, p};
                }
                std::sort(dist.begin(), dist.end());
                for (int j = 0; j < h->ne; j++) {
                    colidx[(size_t)rb * np + j] = dist[j].second;
                    colpos[(size_t)rb * np + dist[j].second] = j;
                }
            }
        };
        int nth = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
        std::vector<std::thread> ths;
        for (int t = 0; t < nth; t++) ths.emplace_back(sort_rb, t, nth);
        for (auto& t : ths) t.join();
    }
    h->d_colidx = (int*)dalloc(h, sizeof(int) * colidx.size());
    if (!h->d_colidx) return fail(h, MOT_EOOM, "device allocation (column order)");
    CK(cudaMemcpy(h->d_colidx, colidx.data(), sizeof(int) * colidx.size(), cudaMemcpyHostToDevice));
    int max_tail = 0;
    // pass 1: validate and mark occupied tiles
    for (int mi = 0; mi < 12; mi++) {
        const mot_lagmat& M = ops->mat[mi];
        const int kind = kMatKind[mi];
        const int fam = kKindFamily[kind];
        const int lagmax = fam == 0 ? h->kmax : fam == 1 ? h->kmax + 1 : h->kmax - 1;
        if (M.nent > 0 && (!M.rowptr || !M.col || !M.k0 || !M.cnt || !M.voff || !M.val))
            return fail(h, MOT_EINVAL, "lag matrix with missing arrays");
        if (M.nent > 0 && M.rowptr[h->ne] != M.nent) return fail(h, MOT_EINVAL, "lag matrix rowptr[ne] != nent");
        const bool tails = (mi == 5 || mi == 11) && M.tail_lag && M.tail_val;
        for (int m = 0; m < h->ne && M.nent > 0; m++) {
            const int rb = h->iperm[m] / T;
            for (int64_t e = M.rowptr[m]; e < M.rowptr[m + 1]; e++) {
                const int n = M.col[e];
                if (n < 0 || n >= h->ne) return fail(h, MOT_EINVAL, "lag matrix column out of range");
                const int cb = colpos[(size_t)rb * np + h->iperm[n]] / T;
                const int k0 = M.k0[e], c = M.cnt[e];
                if (k0 < 0 || c < 0) return fail(h, MOT_EINVAL, "negative lag window");
                for (int k = k0; k < k0 + c; k++) {
                    const double v = M.val[M.voff[e] + (k - k0)];
                    if (!std::isfinite(v)) return fail(h, MOT_EINVAL, "non-finite operator value");
                    if (k > lagmax) {
                        if (fam == 2) continue;  // explicit truncation of A~ (Section V-B-3)
                        if (v != 0.0) return fail(h, MOT_EINVAL, "operator lag beyond its family's range");
                        continue;
                    }
                    if (v == 0.0) continue;
                    size_t kk = key(kind, k, rb, cb);
                    if (id[kk] < 0) id[kk] = -2;
                }
                if (tails) {
                    const int a = M.tail_lag[e];
                    const double v = M.tail_val[e];
                    if (!std::isfinite(v)) return fail(h, MOT_EINVAL, "non-finite tail value");
                    if (a >= 1 && a <= h->kmax - 1 && v != 0.0) {
                        size_t kk = key(9, a, rb, cb);
                        if (id[kk] < 0) id[kk] = -2;
                        max_tail = std::max(max_tail, a);
                    }
                }
            }
        }
    }
    // Tile numbering: row block major, then (kind, lag, column block), so that
    // the tiles of a range of row blocks are contiguous and can be filled on
    // the host and uploaded range by range (the FP64 values of every tile
    // are never held at once). The mixed path keeps FP64 copies of the lag-0
    // tiles only (the dense Q_0 assembly reads them), in a compact numbering;
    // every other tile goes to the device as FP32.
    const bool mixed_tiles = h->opt.precision == MOT_PREC_MIXED && mflag(h, MOT_MIX_HIST32);
    std::vector<int64_t> rb_first(nrb + 1, 0);
    std::vector<int> lag0_slot;  // compact index of a lag-0 tile (mixed path), -1 otherwise
    int64_t nt = 0, n0 = 0;
    for (int rb = 0; rb < nrb; rb++) {
        rb_first[rb] = nt;
        for (int kind = 0; kind < NTK; kind++)
            for (int k = 0; k < L; k++)
                for (int cb = 0; cb < nrb; cb++) {
                    int& v = id[key(kind, k, rb, cb)];
                    if (v != -2) continue;
                    v = (int)nt++;
                    lag0_slot.push_back(k == 0 && kKindFamily[kind] != 3 ? (int)n0++ : -1);
                }
    }
    rb_first[nrb] = nt;
    h->ntiles = nt;
    h->ntiles_fp64 = mixed_tiles ? n0 : nt;
    h->max_tail_lag = max_tail;
    const size_t TT = (size_t)T * T;
    if (mixed_tiles) {
        h->d_tiles = (double*)dalloc(h, sizeof(double) * std::max<int64_t>(1, n0) * TT);
        h->d_tiles32 = (float*)dalloc(h, sizeof(float) * std::max<int64_t>(1, nt) * TT);
        if (!h->d_tiles || !h->d_tiles32) return fail(h, MOT_EOOM, "device allocation (history tiles)");
    } else {
        h->d_tiles = (double*)dalloc(h, sizeof(double) * std::max<int64_t>(1, nt) * TT);
        if (!h->d_tiles) return fail(h, MOT_EOOM, "device allocation (history tiles)");
    }
    // internal rows of every row block
    std::vector<int> tnnz(nt, 0);
    int nth = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    const int64_t batch_tiles = 1 << 18;  // at most 2 GB of FP64 tiles on the host at a time
    std::vector<double> buf;
    std::vector<float> buf32;
    int rb0 = 0;
    while (rb0 < nrb) {
        int rb1 = rb0 + 1;
        while (rb1 < nrb && rb_first[rb1 + 1] - rb_first[rb0] <= batch_tiles) rb1++;
        const int64_t t0 = rb_first[rb0], ntb = rb_first[rb1] - t0;
        buf.assign((size_t)ntb * TT, 0.0);
        // pass 2 over the rows of row blocks [rb0, rb1) (threads split the row blocks)
        auto fill = [&](int tid) {
            for (int mi = 0; mi < 12; mi++) {
                const mot_lagmat& M = ops->mat[mi];
                const int kind = kMatKind[mi];
                const int fam = kKindFamily[kind];
                const int lagmax = fam == 0 ? h->kmax : fam == 1 ? h->kmax + 1 : h->kmax - 1;
                const bool tails = (mi == 5 || mi == 11) && M.tail_lag && M.tail_val;
                if (M.nent == 0) continue;
                for (int rb = rb0 + tid; rb < rb1; rb += nth)
                    for (int p = rb * T; p < std::min(h->ne, rb * T + T); p++) {
                        const int m = h->perm[p];
                        const int r = p - rb * T;
                        for (int64_t e = M.rowptr[m]; e < M.rowptr[m + 1]; e++) {
                            const int q = h->iperm[M.col[e]];
                            const int qs = colpos[(size_t)rb * np + q];
                            const int cb = qs / T, cc = qs - cb * T;
                            for (int k = M.k0[e]; k < M.k0[e] + M.cnt[e] && k <= lagmax; k++) {
                                const double v = M.val[M.voff[e] + (k - M.k0[e])];
                                if (v == 0.0) continue;
                                buf[(size_t)(id[key(kind, k, rb, cb)] - t0) * TT + r * T + cc] += v;
                            }
                            if (tails) {
                                const int a = M.tail_lag[e];
                                const double v = M.tail_val[e];
                                if (a >= 1 && a <= h->kmax - 1 && v != 0.0)
                                    buf[(size_t)(id[key(9, a, rb, cb)] - t0) * TT + r * T + cc] += v;
                            }
                        }
                    }
            }
        };
        {
            std::vector<std::thread> th;
            for (int t = 0; t < nth; t++) th.emplace_back(fill, t);
            for (auto& t : th) t.join();
        }
        for (int64_t t = 0; t < ntb; t++)
            for (size_t e = 0; e < TT; e++) tnnz[t0 + t] += buf[(size_t)t * TT + e] != 0.0;
        if (mixed_tiles) {
            buf32.resize(buf.size());
            for (size_t e = 0; e < buf.size(); e++) buf32[e] = (float)buf[e];
            CK(cudaMemcpy(h->d_tiles32 + (size_t)t0 * TT, buf32.data(), sizeof(float) * buf32.size(),
                          cudaMemcpyHostToDevice));
            for (int64_t t = 0; t < ntb; t++)
                if (lag0_slot[t0 + t] >= 0)
                    CK(cudaMemcpy(h->d_tiles + (size_t)lag0_slot[t0 + t] * TT, buf.data() + (size_t)t * TT,
                                  sizeof(double) * TT, cudaMemcpyHostToDevice));
        } else if (ntb > 0) {
            CK(cudaMemcpy(h->d_tiles + (size_t)t0 * TT, buf.data(), sizeof(double) * buf.size(),
                          cudaMemcpyHostToDevice));
        }
        rb0 = rb1;
    }
    std::vector<double>().swap(buf);
    std::vector<float>().swap(buf32);
    int64_t nz = 0;
    for (int64_t t = 0; t < nt; t++) nz += tnnz[t];
    h->tile_fill = nt ? (double)nz / ((double)nt * T * T) : 0.0;
    std::vector<char> used_hist(nt, 0);
    // task lists
    std::vector<HistTask> th_hist, th_lag0;
    std::vector<int> rb_hist, rb_lag0;
    for (int kind = 0; kind < NTK; kind++)
        for (int k = 0; k < L; k++)
            for (int rb = 0; rb < nrb; rb++)
                for (int cb = 0; cb < nrb; cb++) {
                    int t = id[key(kind, k, rb, cb)];
                    if (t < 0) continue;
                    const int fam = kKindFamily[kind], var = kKindVariant[kind];
                    auto push = [&](int part, int outi) {
                        HistTask tk{t, cb, k, part | (var << 2) | (outi << 4)};
                        if (k == 0 && fam != 3) {
                            if (mixed_tiles) tk.tile = lag0_slot[t];  // the compact FP64 lag-0 tiles
                            th_lag0.push_back(tk);
                            rb_lag0.push_back(rb);
                        } else {
                            th_hist.push_back(tk);
                            rb_hist.push_back(rb);
                            h->hist_nnz_tasks += tnnz[t];
                            if (!used_hist[t]) {
                                used_hist[t] = 1;
                                h->hist_nnz_unique += tnnz[t];
                            }
                        }
                    };
                    if (fam == 0) {
                        push(0, 0);  // A_k l -> s1
                        push(1, 1);  // A_k s -> s2
                    } else if (fam == 1) {
                        push(1, 0);  // A^_k s -> s1
                    } else if (fam == 2) {
                        push(0, 1);  // A~_k l -> s2
                    } else {
                        push(2, 1);  // tail slice * W_a -> s2
                    }
                }
    int nsm = 148;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->dev);
    auto make_list = [&](std::vector<HistTask>& tasks, std::vector<int>& rbs, TaskList& tl) -> int {
        std::vector<int> order(tasks.size());
        std::iota(order.begin(), order.end(), 0);
        std::sort(order.begin(), order.end(), [&](int a, int b) {
            if (rbs[a] != rbs[b]) return rbs[a] < rbs[b];
            const int oa = (tasks[a].code >> 4) & 1, ob = (tasks[b].code >> 4) & 1;
            if (oa != ob) return oa < ob;  // contiguous runs per output target
            if (tasks[a].k != tasks[b].k) return tasks[a].k < tasks[b].k;
            return tasks[a].cb < tasks[b].cb;
        });
        std::vector<HistTask> sorted(tasks.size());
        std::vector<int> srb(tasks.size());
        for (size_t i = 0; i < order.size(); i++) {
            sorted[i] = tasks[order[i]];
            srb[i] = rbs[order[i]];
        }
        const size_t target_chunks = (size_t)4 * nsm;
        const int ch = (int)std::max<size_t>(1, (sorted.size() + target_chunks - 1) / target_chunks);
        std::vector<HistChunk> chunks;
        std::vector<int> cptr(nrb + 1, 0);
        size_t i = 0;
        for (int rb = 0; rb < nrb; rb++) {
            cptr[rb] = (int)chunks.size();
            while (i < sorted.size() && srb[i] == rb) {
                size_t j = i;
                while (j < sorted.size() && srb[j] == rb && (int)(j - i) < ch) j++;
                chunks.push_back(HistChunk{rb, (int)i, (int)(j - i)});
                i = j;
            }
        }
        cptr[nrb] = (int)chunks.size();
        tl.ntasks = (int)sorted.size();
        tl.nchunks = (int)chunks.size();
        tl.tasks = (HistTask*)dalloc(h, sizeof(HistTask) * std::max<size_t>(1, sorted.size()));
        tl.chunks = (HistChunk*)dalloc(h, sizeof(HistChunk) * std::max<size_t>(1, chunks.size()));
        tl.chunk_ptr = (int*)dalloc(h, sizeof(int) * (nrb + 1));
        if (!tl.tasks || !tl.chunks || !tl.chunk_ptr) return fail(h, MOT_EOOM, "device allocation (task list)");
        if (!sorted.empty()) CK(cudaMemcpy(tl.tasks, sorted.data(), sizeof(HistTask) * sorted.size(), cudaMemcpyHostToDevice));
        if (!chunks.empty()) CK(cudaMemcpy(tl.chunks, chunks.data(), sizeof(HistChunk) * chunks.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(tl.chunk_ptr, cptr.data(), sizeof(int) * (nrb + 1), cudaMemcpyHostToDevice));
        return MOT_OK;
    };
    int st;
    if ((st = make_list(th_hist, rb_hist, h->hist)) != MOT_OK) return st;
    if ((st = make_list(th_lag0, rb_lag0, h->lag0)) != MOT_OK) return st;
    if (h->opt.precision == MOT_PREC_MIXED && (h->opt.mixed_flags & MOT_MIX_TC)) {
        if ((st = make_tc_list(h, th_hist, rb_hist, MOT_TC_CHUNK, 0.4)) != MOT_OK) return st;
        h->tc_tasks_host = std::move(th_hist);  // kept for re-chunking by the tuner
        h->tc_rbs_host = std::move(rb_hist);
    }
    return MOT_OK;
}

}  // namespace

namespace {

// Mixed path set-up: dense Q_0 and [M1 | M2] assembled column by column from the
// FP64 product form (64 unit columns per batch), then FP32 copies of them and of
// the history tiles. The FP64 history tiles are released afterwards.
int precompute_mixed(mot_handle* h) {
    const int Bp = 64;
    h->precomputing = true;
    int st = ensure_state(h, Bp);
    if (st != MOT_OK) return st;
    Work W = work_of(h);
    cudaStream_t s = 0;
    const long long n2 = 2LL * h->npad;
    h->d_Q0 = (double*)dalloc(h, sizeof(double) * (size_t)n2 * n2);
    h->d_LF = (double*)dalloc(h, sizeof(double) * (size_t)h->npad * n2);
    h->d_Q0f = (float*)dalloc(h, sizeof(float) * (size_t)n2 * n2);
    h->d_LFf = (float*)dalloc(h, sizeof(float) * (size_t)h->npad * n2);
    const bool h32 = (h->opt.mixed_flags & MOT_MIX_HIST32) != 0;  // FP32 tiles written by build_tiles
    if (!h->d_Q0 || !h->d_LF || !h->d_Q0f || !h->d_LFf || (h32 && !h->d_tiles32))
        return fail(h, MOT_EOOM, "device allocation (mixed-precision operators)");
    CK(cudaMemsetAsync(h->d_cg_iters, 0, 2 * sizeof(int), s));
    for (long long J0 = 0; J0 < n2; J0 += Bp) {
        launch_unit_cols(h, J0, n2, W.x, s);
        apply_q0(h, W, W.x, W.w, s);
        launch_scatter_cols(h, J0, n2, W.w, h->d_Q0, n2, s);
    }
    for (long long Q0 = 0; Q0 < n2; Q0 += Bp) {
        launch_unit_lf(h, Q0, n2, W.rho1, W.rho2, s);
        left_factor(h, W, W.rho1, W.rho2, W.b, s);
        launch_scatter_lf(h, Q0, n2, W.b, h->d_LF, n2, s);
    }
    launch_d2f(h, (size_t)n2 * n2, h->d_Q0, h->d_Q0f, s);
    launch_d2f(h, (size_t)h->npad * n2, h->d_LF, h->d_LFf, s);
    if (h->opt.mixed_flags & MOT_MIX_PRECOND) {
        // GMRES preconditioner: Q_0^{-1} by LU with partial pivoting (FP64), kept in FP32
        double* lu = (double*)dalloc(h, sizeof(double) * (size_t)n2 * n2);
        double* inv = (double*)dalloc(h, sizeof(double) * (size_t)n2 * n2);
        int* piv = (int*)dalloc(h, sizeof(int) * (size_t)(n2 + 1));
        h->d_Minvf = (float*)dalloc(h, sizeof(float) * (size_t)n2 * n2);
        if (!lu || !inv || !piv || !h->d_Minvf) return fail(h, MOT_EOOM, "device allocation (Q_0 factorisation)");
        CK(cudaMemcpyAsync(lu, h->d_Q0, sizeof(double) * (size_t)n2 * n2, cudaMemcpyDeviceToDevice, s));
        dense_pad_identity(h, (int)n2, h->ne, lu, s);
        const int bad = dense_lu(h, (int)n2, lu, piv, piv + n2, s);
        if (bad > 0) {
            cudaFree(lu);
            cudaFree(inv);
            cudaFree(piv);
            return fail(h, MOT_EINVAL, "Q_0 is singular to working precision (LU pivot breakdown)");
        }
        dense_inverse_from_lu(h, (int)n2, lu, piv, inv, s);
        launch_d2f(h, (size_t)n2 * n2, inv, h->d_Minvf, s);
        if (emu_ok(h)) {  // 4-slice copy for the tensor-core products of the FP32 solves
            CK(cudaDeviceSynchronize());
            if ((st = emu_prepare(h, inv, (int)n2, (int)n2, &h->emu_Minv, 4)) != MOT_OK) return st;
        }
        CK(cudaDeviceSynchronize());
        cudaFree(lu);
        cudaFree(inv);
        cudaFree(piv);
        h->device_bytes -= (int64_t)(2 * sizeof(double) * (size_t)n2 * n2 + sizeof(int) * (size_t)(n2 + 1));
    }
    {
        // preconditioner of the FP64 CG behind P^Sigma: (Sigma^T Sigma + 11^T/N_f)^{-1}, which is the
        // pseudo-inverse on the range of the face Laplacian (connected surface), kept in FP32
        const int npd = (h->nf + 63) / 64 * 64;
        double* A = (double*)dalloc(h, sizeof(double) * (size_t)npd * npd);
        double* inv = (double*)dalloc(h, sizeof(double) * (size_t)npd * npd);
        int* piv = (int*)dalloc(h, sizeof(int) * (size_t)(npd + 1));
        h->d_Lfinvf = (float*)dalloc(h, sizeof(float) * (size_t)npd * npd);
        if (!A || !inv || !piv || !h->d_Lfinvf) return fail(h, MOT_EOOM, "device allocation (Laplacian factorisation)");
        dense_lap_plus_j(h, h->Lf, npd, A, s);
        const int bad = dense_lu(h, npd, A, piv, piv + npd, s);
        if (bad == 0) {
            dense_inverse_from_lu(h, npd, A, piv, inv, s);
            launch_d2f(h, (size_t)npd * npd, inv, h->d_Lfinvf, s);
            h->nfpd = npd;
        }
        CK(cudaDeviceSynchronize());
        cudaFree(A);
        cudaFree(inv);
        cudaFree(piv);
        h->device_bytes -= (int64_t)(2 * sizeof(double) * (size_t)npd * npd + sizeof(int) * (size_t)(npd + 1));
        if (bad != 0) {  // not connected: keep the plain CG
            cudaFree(h->d_Lfinvf);
            h->d_Lfinvf = nullptr;
        }
    }
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    int it[2];
    CK(cudaMemcpy(it, h->d_cg_iters, 2 * sizeof(int), cudaMemcpyDeviceToHost));
    free_state(h);
    h->precomputing = false;
    if (it[1] > 0) return fail(h, MOT_ENOCONV, "a CG solve did not converge while assembling the dense operators");
    if (emu_ok(h)) {  // slices of Q_0 and [M1 | M2] for the emulated products
        if ((st = emu_prepare(h, h->d_Q0, 2 * h->npad, 2 * h->npad, &h->emu_Q0, 6)) != MOT_OK) return st;
        if ((st = emu_prepare(h, h->d_LF, h->npad, 2 * h->npad, &h->emu_LF, 6)) != MOT_OK) return st;
        if (mflag(h, MOT_MIX_Q032) &&
            (st = emu_prepare(h, h->d_Q0, 2 * h->npad, 2 * h->npad, &h->emu_Q0s, 4)) != MOT_OK)
            return st;
        CK(cudaDeviceSynchronize());
    }
    if (h32) {  // the FP64 lag-0 tiles (the dense Q_0 assembly's input) are no longer read
        cudaFree(h->d_tiles);
        h->device_bytes -=
            (int64_t)(sizeof(double) * (size_t)std::max<int64_t>(1, h->ntiles_fp64) * MOT_TILE * MOT_TILE);
        h->d_tiles = nullptr;
    }
    return MOT_OK;
}

// FP64 path with fp64_precond: Q_0^{-1} in FP64 as the right preconditioner of
// GMRES. Q_0 is assembled column by column from the FP64 product form (64 unit
// columns per batch), factorised by LU with partial pivoting and inverted; the
// padded rows carry the identity.
int precompute_fp64_precond(mot_handle* h) {
    const int Bp = 64;
    h->precomputing = true;
    int st = ensure_state(h, Bp);
    if (st != MOT_OK) return st;
    Work W = work_of(h);
    cudaStream_t s = 0;
    const long long n2 = 2LL * h->npad;
    double* q0 = (double*)dalloc(h, sizeof(double) * (size_t)n2 * n2);
    int* piv = (int*)dalloc(h, sizeof(int) * (size_t)(n2 + 1));
    h->d_Minv64 = (double*)dalloc(h, sizeof(double) * (size_t)n2 * n2);
    if (!q0 || !piv || !h->d_Minv64) return fail(h, MOT_EOOM, "device allocation (FP64 Q_0 factorisation)");
    CK(cudaMemsetAsync(h->d_cg_iters, 0, 2 * sizeof(int), s));
    for (long long J0 = 0; J0 < n2; J0 += Bp) {
        launch_unit_cols(h, J0, n2, W.x, s);
        apply_q0(h, W, W.x, W.w, s);
        launch_scatter_cols(h, J0, n2, W.w, q0, n2, s);
    }
    dense_pad_identity(h, (int)n2, h->ne, q0, s);
    const int bad = dense_lu(h, (int)n2, q0, piv, piv + n2, s);
    if (bad == 0) dense_inverse_from_lu(h, (int)n2, q0, piv, h->d_Minv64, s);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    int it[2];
    CK(cudaMemcpy(it, h->d_cg_iters, 2 * sizeof(int), cudaMemcpyDeviceToHost));
    cudaFree(q0);
    cudaFree(piv);
    h->device_bytes -= (int64_t)(sizeof(double) * (size_t)n2 * n2 + sizeof(int) * (size_t)(n2 + 1));
    free_state(h);
    h->precomputing = false;
    if (bad > 0) return fail(h, MOT_EINVAL, "Q_0 is singular to working precision (LU pivot breakdown)");
    if (it[1] > 0) return fail(h, MOT_ENOCONV, "a CG solve did not converge while assembling Q_0");
    return MOT_OK;
}

// FP64 path with fp64_direct: dense FP64 inverses of the Gram matrix and of
// the two graph Laplacians (plus 11^T/N), formed once by LU with partial
// pivoting, so the left factor and the projectors are exact to rounding
// instead of to the CG tolerance. tg: the Gram matrix's triplets in the
// internal order.
int prepare_fp64_direct(mot_handle* h, const std::vector<std::tuple<int, int, double>>& tg) {
    cudaStream_t s = 0;
    const int np = h->npad;
    {  // G^{-1}: the leading npad x npad block of the inverse of [[G, 0], [0, I]] (a multiple of 64)
        const int gpd = (np + 63) / 64 * 64;
        std::vector<double> g((size_t)gpd * gpd, 0.0);
        for (const auto& t : tg) g[(size_t)std::get<0>(t) * gpd + std::get<1>(t)] += std::get<2>(t);
        for (int i = h->ne; i < gpd; i++) g[(size_t)i * gpd + i] = 1.0;
        double* A = (double*)dalloc(h, sizeof(double) * (size_t)gpd * gpd);
        double* inv = (double*)dalloc(h, sizeof(double) * (size_t)gpd * gpd);
        int* piv = (int*)dalloc(h, sizeof(int) * (size_t)(gpd + 1));
        h->d_Ginv64 = (double*)dalloc(h, sizeof(double) * (size_t)np * np);
        if (!A || !inv || !piv || !h->d_Ginv64) return fail(h, MOT_EOOM, "device allocation (dense G inverse)");
        CK(cudaMemcpy(A, g.data(), sizeof(double) * g.size(), cudaMemcpyHostToDevice));
        const int bad = dense_lu(h, gpd, A, piv, piv + gpd, s);
        if (bad == 0) {
            dense_inverse_from_lu(h, gpd, A, piv, inv, s);
            CK(cudaMemcpy2DAsync(h->d_Ginv64, sizeof(double) * np, inv, sizeof(double) * gpd, sizeof(double) * np, np,
                                 cudaMemcpyDeviceToDevice, s));
        }
        CK(cudaDeviceSynchronize());
        cudaFree(A);
        cudaFree(inv);
        cudaFree(piv);
        h->device_bytes -= (int64_t)(2 * sizeof(double) * (size_t)gpd * gpd + sizeof(int) * (size_t)(gpd + 1));
        if (bad != 0) return fail(h, MOT_EINVAL, "G is singular to working precision (LU pivot breakdown)");
    }
    auto lap = [&](const DCsr& L, int n, double** out, int* npd_out) -> int {
        const int npd = (n + 63) / 64 * 64;
        double* A = (double*)dalloc(h, sizeof(double) * (size_t)npd * npd);
        int* piv = (int*)dalloc(h, sizeof(int) * (size_t)(npd + 1));
        *out = (double*)dalloc(h, sizeof(double) * (size_t)npd * npd);
        if (!A || !piv || !*out) return fail(h, MOT_EOOM, "device allocation (dense Laplacian inverse)");
        dense_lap_plus_j(h, L, npd, A, s);
        const int bad = dense_lu(h, npd, A, piv, piv + npd, s);
        if (bad == 0) dense_inverse_from_lu(h, npd, A, piv, *out, s);
        CK(cudaDeviceSynchronize());
        cudaFree(A);
        cudaFree(piv);
        h->device_bytes -= (int64_t)(sizeof(double) * (size_t)npd * npd + sizeof(int) * (size_t)(npd + 1));
        if (bad != 0) return fail(h, MOT_EINVAL, "a graph Laplacian plus 11^T/N is singular (surface not connected?)");
        *npd_out = npd;
        return MOT_OK;
    };
    int st;
    if ((st = lap(h->Lf, h->nf, &h->d_Lfinv64, &h->dfpd)) != MOT_OK) return st;
    if ((st = lap(h->Lv, h->nv, &h->d_Lvinv64, &h->dvpd)) != MOT_OK) return st;
    const size_t cmax = 4 * MOT_MAX_B;  // widest block projected: the left factor's 4B columns
    const size_t rows = (size_t)std::max(h->dfpd, h->dvpd);
    h->d_dir_r = (double*)dalloc(h, sizeof(double) * rows * cmax);
    h->d_dir_z = (double*)dalloc(h, sizeof(double) * rows * cmax);
    h->d_dir_sc = (double*)dalloc(h, sizeof(double) * cmax);
    if (!h->d_dir_r || !h->d_dir_z || !h->d_dir_sc) return fail(h, MOT_EOOM, "device allocation (direct solves)");
    return MOT_OK;
}

}  // namespace

MOT_API int mot_load_operators(mot_handle* h, const mot_operators* ops) {
    if (!h) return MOT_EINVAL;
    if (h->loaded) return fail(h, MOT_ESTATE, "operators already loaded");
    if (!ops || !ops->T0s || !ops->T0h || !ops->g_rowptr || !ops->g_col || !ops->g_val || !ops->rhs_x ||
        !ops->rhs_wf || ops->nq <= 0)
        return fail(h, MOT_EINVAL, "missing operator arrays");
    CK(cudaSetDevice(h->dev));
    const int ne = h->ne, np = h->npad;
    // static operators, permuted and zero padded
    std::vector<double> a((size_t)np * np, 0.0), b((size_t)np * np, 0.0);
    for (int p = 0; p < ne; p++)
        for (int q = 0; q < ne; q++) {
            const size_t src = (size_t)h->perm[p] * ne + h->perm[q];
            const double x = ops->T0s[src], y = ops->T0h[src];
            if (!std::isfinite(x) || !std::isfinite(y)) return fail(h, MOT_EINVAL, "non-finite static operator");
            a[(size_t)p * np + q] = x;
            b[(size_t)p * np + q] = y;
        }
    h->d_T0s = (double*)dalloc(h, sizeof(double) * a.size());
    h->d_T0h = (double*)dalloc(h, sizeof(double) * b.size());
    if (!h->d_T0s || !h->d_T0h) return fail(h, MOT_EOOM, "device allocation (static operators)");
    CK(cudaMemcpy(h->d_T0s, a.data(), sizeof(double) * a.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_T0h, b.data(), sizeof(double) * b.size(), cudaMemcpyHostToDevice));
    // Gram matrix and transpose in the internal order
    std::vector<std::tuple<int, int, double>> tg, tgt;
    if (ops->g_rowptr[0] != 0) return fail(h, MOT_EINVAL, "G rowptr[0] != 0");
    for (int m = 0; m < ne; m++)
        for (int64_t e = ops->g_rowptr[m]; e < ops->g_rowptr[m + 1]; e++) {
            const int n = ops->g_col[e];
            const double v = ops->g_val[e];
            if (n < 0 || n >= ne) return fail(h, MOT_EINVAL, "G column out of range");
            if (!std::isfinite(v)) return fail(h, MOT_EINVAL, "non-finite G value");
            tg.emplace_back(h->iperm[m], h->iperm[n], v);
            tgt.emplace_back(h->iperm[n], h->iperm[m], v);
        }
    int st;
    HostCsr G = csr_from_triplets(ne, ne, tg), Gt = csr_from_triplets(ne, ne, tgt);
    if ((st = upload_csr(h, G, h->G)) != MOT_OK) return st;
    if ((st = upload_csr(h, Gt, h->Gt)) != MOT_OK) return st;
    if (h->opt.precision == MOT_PREC_FP64 && h->opt.fp64_direct && (st = prepare_fp64_direct(h, tg)) != MOT_OK)
        return st;
    // RHS quadrature table
    h->nq = ops->nq;
    std::vector<double> x((size_t)np * h->nq * 3, 0.0), wf((size_t)np * h->nq * 3, 0.0);
    for (int p = 0; p < ne; p++) {
        const size_t s = (size_t)h->perm[p] * h->nq * 3, d = (size_t)p * h->nq * 3;
        for (int i = 0; i < h->nq * 3; i++) {
            x[d + i] = ops->rhs_x[s + i];
            wf[d + i] = ops->rhs_wf[s + i];
            if (!std::isfinite(x[d + i]) || !std::isfinite(wf[d + i])) return fail(h, MOT_EINVAL, "non-finite RHS table");
        }
    }
    h->d_rhs_x = (double*)dalloc(h, sizeof(double) * x.size());
    h->d_rhs_wf = (double*)dalloc(h, sizeof(double) * wf.size());
    if (!h->d_rhs_x || !h->d_rhs_wf) return fail(h, MOT_EOOM, "device allocation (RHS table)");
    CK(cudaMemcpy(h->d_rhs_x, x.data(), sizeof(double) * x.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_rhs_wf, wf.data(), sizeof(double) * wf.size(), cudaMemcpyHostToDevice));
    h->tc_bulk = h->opt.precision == MOT_PREC_MIXED && mflag(h, MOT_MIX_TC) && mflag(h, MOT_MIX_TCBULK);
    if ((st = build_tiles(h, ops)) != MOT_OK) return st;
    if (h->opt.precision == MOT_PREC_MIXED && (st = precompute_mixed(h)) != MOT_OK) return st;
    if (h->opt.precision == MOT_PREC_FP64 && h->opt.fp64_precond && (st = precompute_fp64_precond(h)) != MOT_OK)
        return st;
    h->loaded = true;
    return MOT_OK;
}

MOT_API int mot_set_frequencies(mot_handle* h, int n_freq, const double* omega) {
    if (!h) return MOT_EINVAL;
    if (h->step != 0 || h->B != 0) return fail(h, MOT_ESTATE, "set frequencies before the first step");
    if (n_freq < 0 || (n_freq > 0 && !omega)) return fail(h, MOT_EINVAL, "bad frequency list");
    CK(cudaSetDevice(h->dev));
    if (h->d_omega) cudaFree(h->d_omega);
    h->d_omega = nullptr;
    h->nfreq = n_freq;
    h->omega.assign(omega, omega + n_freq);
    for (double w : h->omega)
        if (!std::isfinite(w) || w < 0) return fail(h, MOT_EINVAL, "frequencies must be finite and >= 0");
    if (n_freq > 0) {
        h->d_omega = (double*)dalloc(h, sizeof(double) * n_freq);
        if (!h->d_omega) return fail(h, MOT_EOOM, "device allocation (frequencies)");
        CK(cudaMemcpy(h->d_omega, omega, sizeof(double) * n_freq, cudaMemcpyHostToDevice));
    }
    return MOT_OK;
}

namespace {

// mot_step in two halves around its history contraction: step_begin checks
// the call, uploads the waves and runs the STEP_INPUTS phase (with `phases`
// = STEP_INPUTS | STEP_HISTORY also the history); step_end runs STEP_SOLVE
// and returns w_i.
int step_begin(mot_handle* h, const mot_wave* waves, int B, cudaStream_t s, int phases) {
    if (!h) return MOT_EINVAL;
    if (!h->loaded) return fail(h, MOT_ESTATE, "mot_load_operators must come first");
    if (B < 1 || B > MOT_MAX_B || !waves) return fail(h, MOT_EINVAL, "B must be in [1, 64] with B waves");
    int st;
    if ((st = check_waves(h, waves, B)) != MOT_OK) return st;
    CK(cudaSetDevice(h->dev));
    if ((st = ensure_state(h, B)) != MOT_OK) return st;
    if ((st = upload_waves(h, waves, B, s)) != MOT_OK) return st;
    return do_step(h, s, phases);
}

int step_end(mot_handle* h, int B, double* w_out, cudaStream_t s) {
    int st = do_step(h, s, STEP_SOLVE);
    if (st != MOT_OK && st != MOT_ENOCONV) return st;
    CK(cudaEventRecord(h->ev_state, s));
    if (w_out) {
        Work W = work_of(h);
        if (is_device_ptr(w_out)) {
            launch_pack_w(h, W.x, w_out, s);
        } else {
            launch_pack_w(h, W.x, W.tmp, s);
            CK(cudaMemcpyAsync(w_out, W.tmp, sizeof(double) * (size_t)B * 2 * h->ne, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
        }
        CK(cudaGetLastError());
    }
    return st;
}

}  // namespace

MOT_API int mot_step(mot_handle* h, const mot_wave* waves, int B, double* w_out, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const int st = step_begin(h, waves, B, s, STEP_INPUTS | STEP_HISTORY);
    if (st != MOT_OK) return st;
    return step_end(h, B, w_out, s);
}

MOT_API int mot_run(mot_handle* h, int n_steps, const mot_wave* waves, int B, double* w_out, void* stream) {
    if (!h) return MOT_EINVAL;
    if (n_steps < 0) return fail(h, MOT_EINVAL, "n_steps < 0");
    int worst = MOT_OK;
    const bool dev = w_out && is_device_ptr(w_out);
    for (int i = 0; i < n_steps; i++) {
        double* dst = w_out ? w_out + (size_t)i * B * 2 * h->ne : nullptr;
        (void)dev;
        int st = mot_step(h, waves, B, dst, stream);
        if (st == MOT_ENOCONV) worst = st;
        else if (st != MOT_OK) return st;
    }
    return worst;
}

namespace {

// Reusable barrier of a fixed number of host threads.
class HostBarrier {
   public:
    explicit HostBarrier(int n) : n_(n) {}
    void wait() {
        std::unique_lock<std::mutex> lk(m_);
        const long gen = gen_;
        if (++count_ == n_) {
            count_ = 0;
            gen_++;
            cv_.notify_all();
        } else {
            cv_.wait(lk, [&] { return gen_ != gen; });
        }
    }

   private:
    std::mutex m_;
    std::condition_variable cv_;
    int n_, count_ = 0;
    long gen_ = 0;
};

// Grows the chunk-sum buffer of h to the current tensor-core list.
int fit_partial(mot_handle* h) {
    const size_t need = sizeof(double) * (size_t)std::max(1, h->hist_tc_list.nchunks) * 2 * MOT_TILE * 2 * h->B;
    if (need <= h->partial_bytes) return MOT_OK;
    cudaFree(h->d_partial);
    h->device_bytes -= (int64_t)h->partial_bytes;
    h->d_partial = (double*)dalloc(h, need);
    if (!h->d_partial) return fail(h, MOT_EOOM, "device allocation (history chunk sums)");
    h->partial_bytes = need;
    return MOT_OK;
}

// Autotuner of the tensor-core history for handles marched together (one
// launch serves all of them): every candidate (tasks per chunk, lags per L2
// range, pipeline stages and tasks per stage, epilogue warps) is applied,
// launched once to warm up and three times timed with CUDA events on s; the
// fastest (median) is kept. The launches
// read the current march state and write only the chunk sums and the history
// sums of the work area, which every step recomputes before use.
int tune_tc(mot_handle* const* hs, int n, cudaStream_t s) {
    std::vector<double*> s1(n), s2(n);
    int max_npad = 0;
    for (int k = 0; k < n; k++) {
        Work W = work_of(hs[k]);
        s1[k] = W.s1;
        s2[k] = W.s2;
        max_npad = std::max(max_npad, hs[k]->npad);
    }
    const bool bulk = hs[0]->tc_bulk;
    float best = 1e30f;
    int bcap = MOT_TC_CHUNK, bns = 0, bepi = 4, btp = 1;
    double blf = 0.4;
    const int caps[] = {256, 512, 1024};
    const double fracs[] = {0.2, 0.4, 0.8};
    for (int cap : caps)
        for (double lf : fracs) {
            int st;
            for (int k = 0; k < n; k++) {
                if ((st = make_tc_list(hs[k], hs[k]->tc_tasks_host, hs[k]->tc_rbs_host, cap, lf)) != MOT_OK) return st;
                if (!hs[k]->hist_tc_list.packed) return fail(hs[k], MOT_EINVAL, "tensor-core list not available");
                if ((st = fit_partial(hs[k])) != MOT_OK) return st;
            }
            int listcap = 1;
            for (int k = 0; k < n; k++) listcap = std::max(listcap, hs[k]->hist_tc_list.cap);
            const int cfgs[][2] = {{4, 1}, {5, 1}, {2, 2}, {3, 2}};  // (stages, tasks per stage)
            for (const auto& cf : cfgs)
                for (int epi = 4; epi <= 8; epi += 4) {
                    const int ns = cf[0], tp = cf[1];
                    if (!history_tc_config_fits(max_npad, bulk, listcap, ns, tp)) continue;
                    for (int k = 0; k < n; k++) {
                        hs[k]->tc_stages = ns;
                        hs[k]->tc_tps = tp;
                        hs[k]->tc_epi = epi;
                    }
                    launch_history_tc_many(hs, n, s1.data(), s2.data(), s, false);
                    float t[3];
                    for (int r = 0; r < 3; r++) t[r] = launch_history_tc_many(hs, n, s1.data(), s2.data(), s, true);
                    std::sort(t, t + 3);
                    if (cudaGetLastError() != cudaSuccess)
                        return fail(hs[0], MOT_ECUDA, "mot_tune: trial launch failed");
                    if (t[1] < best) {
                        best = t[1];
                        bcap = cap;
                        blf = lf;
                        bns = ns;
                        btp = tp;
                        bepi = epi;
                    }
                }
        }
    for (int k = 0; k < n; k++) {
        int st;
        if ((st = make_tc_list(hs[k], hs[k]->tc_tasks_host, hs[k]->tc_rbs_host, bcap, blf)) != MOT_OK) return st;
        if ((st = fit_partial(hs[k])) != MOT_OK) return st;
        hs[k]->tc_stages = bns;
        hs[k]->tc_tps = btp;
        hs[k]->tc_epi = bepi;
        hs[k]->tc_tuned = true;
        hs[k]->tc_tune_ms = best;
    }
    CK_H(hs[0], cudaStreamSynchronize(s));
    return MOT_OK;
}

}  // namespace

MOT_API int mot_tune(mot_handle* const* hs, int n, void* stream) {
    if (n < 1 || n > MOT_TC_MAX_JOBS || !hs) return MOT_EINVAL;
    std::vector<const mot_handle*> seen(hs, hs + n);
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end() || !seen[0]) return MOT_EINVAL;
    for (int k = 0; k < n; k++) {
        mot_handle* h = hs[k];
        if (!h->hist_tc || h->step < 1)
            return fail(h, MOT_ESTATE, "mot_tune: needs handles on the tensor-core history that have taken a step");
        if (h->tc_bulk != hs[0]->tc_bulk || h->dev != hs[0]->dev)
            return fail(h, MOT_EINVAL, "mot_tune: handles of one kernel form on one device");
    }
    CK_H(hs[0], cudaSetDevice(hs[0]->dev));
    return tune_tc(hs, n, (cudaStream_t)stream);
}

MOT_API int mot_set_tc_config(mot_handle* h, int cap, double lag_frac, int stages, int tasks_per_stage,
                              int epilogue_warps) {
    if (!h) return MOT_EINVAL;
    if (!h->hist_tc || h->step < 1)
        return fail(h, MOT_ESTATE, "mot_set_tc_config: needs a handle on the tensor-core history that has taken a step");
    if (cap < 1 || cap > MOT_TC_CHUNK || !(lag_frac > 0.0 && lag_frac <= 1.0) ||
        (epilogue_warps != 4 && epilogue_warps != 8))
        return fail(h, MOT_EINVAL, "mot_set_tc_config: configuration out of range");
    CK_H(h, cudaSetDevice(h->dev));
    int st;
    if ((st = make_tc_list(h, h->tc_tasks_host, h->tc_rbs_host, cap, lag_frac)) != MOT_OK) return st;
    if (!h->hist_tc_list.packed) return fail(h, MOT_EINVAL, "tensor-core list not available");
    if (!history_tc_config_fits(h->npad, h->tc_bulk, h->hist_tc_list.cap, stages, tasks_per_stage))
        return fail(h, MOT_EINVAL, "mot_set_tc_config: stages x tasks per stage do not fit in shared memory");
    if ((st = fit_partial(h)) != MOT_OK) return st;
    h->tc_stages = stages;
    h->tc_tps = tasks_per_stage;
    h->tc_epi = epilogue_warps;
    h->tc_tuned = false;
    h->tc_tune_ms = 0;
    return MOT_OK;
}

MOT_API int mot_run_many(mot_handle* const* hs, int n, int n_steps, const mot_wave* const* waves, const int* B,
                         double* const* w_out, void* stream) {
    if (n < 0 || n_steps < 0) return MOT_EINVAL;
    if (n == 0) return MOT_OK;
    if (!hs || !waves || !B) return MOT_EINVAL;
    {
        std::vector<const mot_handle*> seen(hs, hs + n);
        std::sort(seen.begin(), seen.end());
        if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) return MOT_EINVAL;
        for (int i = 0; i < n; i++)
            if (!hs[i] || !waves[i]) return MOT_EINVAL;
    }
    cudaStream_t user = (cudaStream_t)stream;
    std::vector<int> st(n, MOT_OK);
    // march state of every scatterer (it decides which run the tensor-core history)
    for (int i = 0; i < n; i++) {
        mot_handle* h = hs[i];
        if (!h->loaded) return fail(h, MOT_ESTATE, "mot_load_operators must come first");
        if (B[i] < 1 || B[i] > MOT_MAX_B) return fail(h, MOT_EINVAL, "B must be in [1, 64] with B waves");
        if (cudaSetDevice(h->dev) != cudaSuccess) return fail(h, MOT_ECUDA, "cudaSetDevice");
        int e = ensure_state(h, B[i]);
        if (e != MOT_OK) return e;
    }
    // the group whose history contractions run as one launch per step: the
    // scatterers on the tensor-core history in the first one's form and device
    std::vector<int> group;
    for (int i = 0; i < n; i++) {
        mot_handle* h = hs[i];
        if (h->hist_tc && (group.empty() || (h->tc_bulk == hs[group[0]]->tc_bulk && h->dev == hs[group[0]]->dev)) &&
            (int)group.size() < MOT_TC_MAX_JOBS)
            group.push_back(i);
    }
    if (group.size() < 2) group.clear();
    std::vector<int> slot(n, -1);
    for (size_t g = 0; g < group.size(); g++) slot[group[g]] = (int)g;
    const int ng = (int)group.size();
    // fork: every scatterer's stream waits for the work queued on `stream`
    cudaEvent_t fork = nullptr;
    {
        mot_handle* h0 = hs[0];
        cudaError_t e = cudaSetDevice(h0->dev);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(fork, user);
        if (e != cudaSuccess) {
            if (fork) cudaEventDestroy(fork);
            return cuda_fail(h0, e, "mot_run_many: fork event");
        }
    }
    std::vector<cudaEvent_t> joins(n, nullptr), ev_in(ng, nullptr);
    cudaEvent_t ev_hist = nullptr;
    cudaStream_t gs = nullptr;  // stream of the group's history launches
    if (ng > 0) {
        cudaError_t e = cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(gs, fork, 0);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_hist, cudaEventDisableTiming);
        for (int g = 0; g < ng && e == cudaSuccess; g++) e = cudaEventCreateWithFlags(&ev_in[g], cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(hs[0], e, "mot_run_many: group set-up");
    }
    HostBarrier bar(std::max(1, ng));
    std::vector<char> gfail(ng, 0);
    int group_status = MOT_OK;
    // the group's history of the coming step, by the first member's thread
    auto group_history = [&]() {
        std::vector<mot_handle*> hm;
        std::vector<double*> s1, s2;
        bool full = true;
        for (int g = 0; g < ng; g++) {
            mot_handle* h = hs[group[g]];
            if (gfail[g] || h->step + 1 < 2) continue;
            cudaStreamWaitEvent(gs, ev_in[g], 0);
            Work W = work_of(h);
            hm.push_back(h);
            s1.push_back(W.s1);
            s2.push_back(W.s2);
            full = full && h->step + 1 > h->K;
        }
        if (!hm.empty()) {
            // tuned once, at the first step that contracts every member's full history
            bool tuned = true;
            for (mot_handle* h : hm) tuned = tuned && h->tc_tuned;
            if (full && !tuned && (int)hm.size() == ng) {
                const int t = tune_tc(hm.data(), (int)hm.size(), gs);
                if (t != MOT_OK) group_status = t;
            }
            const bool timed = full && hm[0]->opt.timing;
            const float ms = launch_history_tc_many(hm.data(), (int)hm.size(), s1.data(), s2.data(), gs, timed);
            if (timed)
                for (mot_handle* h : hm) {
                    h->timed_ms += ms;
                    h->timed_launches++;
                }
        }
        cudaEventRecord(ev_hist, gs);
    };
    auto march = [&](int i) {
        mot_handle* h = hs[i];
        if (cudaSetDevice(h->dev) != cudaSuccess) {
            st[i] = fail(h, MOT_ECUDA, "cudaSetDevice");
            if (slot[i] < 0) return;
        }
        cudaStream_t s = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, fork, 0);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&joins[i], cudaEventDisableTiming);
        if (e != cudaSuccess && st[i] == MOT_OK) st[i] = cuda_fail(h, e, "mot_run_many: stream set-up");
        const int g = slot[i];
        if (g < 0) {
            if (st[i] == MOT_OK) st[i] = mot_run(h, n_steps, waves[i], B[i], w_out ? w_out[i] : nullptr, s);
        } else {
            // lock step with the group: inputs, one history launch for all, solve
            bool ok = st[i] == MOT_OK;
            int worst = MOT_OK;
            double* out = w_out ? w_out[i] : nullptr;
            for (int k = 0; k < n_steps; k++) {
                if (ok) {
                    const int a = step_begin(h, waves[i], B[i], s, STEP_INPUTS);
                    if (a != MOT_OK || cudaEventRecord(ev_in[g], s) != cudaSuccess) {
                        st[i] = a != MOT_OK ? a : fail(h, MOT_ECUDA, "mot_run_many: event");
                        ok = false;
                    }
                }
                gfail[g] = !ok;
                bar.wait();
                if (g == 0) group_history();
                bar.wait();
                if (ok) {
                    cudaStreamWaitEvent(s, ev_hist, 0);
                    double* dst = out ? out + (size_t)k * B[i] * 2 * h->ne : nullptr;
                    const int r = step_end(h, B[i], dst, s);
                    if (r == MOT_ENOCONV) {
                        worst = MOT_ENOCONV;
                    } else if (r != MOT_OK) {
                        st[i] = r;
                        ok = false;
                    }
                }
            }
            if (ok) st[i] = worst;
        }
        if (joins[i]) {
            e = cudaEventRecord(joins[i], s);  // the join point, recorded whatever the status
            if (e != cudaSuccess && st[i] == MOT_OK) st[i] = cuda_fail(h, e, "mot_run_many: join event");
        }
        if (s) cudaStreamDestroy(s);  // released once its work completes
    };
    std::vector<std::thread> th;
    th.reserve(n > 0 ? n - 1 : 0);
    for (int i = 1; i < n; i++) th.emplace_back(march, i);
    march(0);
    for (auto& t : th) t.join();
    // join: later work on `stream` waits for every scatterer
    cudaSetDevice(hs[0]->dev);
    for (int i = 0; i < n; i++)
        if (joins[i]) {
            cudaStreamWaitEvent(user, joins[i], 0);
            cudaEventDestroy(joins[i]);
        }
    if (gs) {
        cudaStreamSynchronize(gs);
        cudaStreamDestroy(gs);
        cudaEventDestroy(ev_hist);
        for (auto ev : ev_in) cudaEventDestroy(ev);
    }
    cudaEventDestroy(fork);
    if (group_status != MOT_OK) return group_status;
    int worst = MOT_OK;
    for (int i = 0; i < n; i++) {
        if (st[i] != MOT_OK && st[i] != MOT_ENOCONV) return st[i];
        if (st[i] == MOT_ENOCONV) worst = MOT_ENOCONV;
    }
    return worst;
}

MOT_API int mot_get_currents(mot_handle* h, double* out) {
    if (!h || !out) return MOT_EINVAL;
    if (!h->d_cur || h->step == 0) return fail(h, MOT_ESTATE, "no step taken yet");
    CK(cudaSetDevice(h->dev));
    CK(cudaStreamWaitEvent(0, h->ev_state, 0));  // after the last step, on whatever stream it ran
    Work W = work_of(h);
    const size_t n = (size_t)h->B * 4 * h->ne;
    if (is_device_ptr(out)) {
        launch_pack_cur(h, out, 0);
    } else {
        launch_pack_cur(h, W.Y4, 0);
        CK(cudaMemcpy(out, W.Y4, sizeof(double) * n, cudaMemcpyDeviceToHost));
    }
    CK(cudaDeviceSynchronize());
    return MOT_OK;
}

MOT_API int mot_fields(mot_handle* h, const mot_wave* waves, int n_dir, const double* dirs, double* E_out) {
    if (!h || !E_out || (n_dir > 0 && !dirs)) return MOT_EINVAL;
    if (!h->d_dft || h->nfreq == 0) return fail(h, MOT_ESTATE, "no Fourier sums: call mot_set_frequencies and step");
    (void)waves;
    CK(cudaSetDevice(h->dev));
    double* dd = (double*)dalloc(h, sizeof(double) * 3 * std::max(1, n_dir));
    double* de = (double*)dalloc(h, sizeof(double) * (size_t)h->B * h->nfreq * std::max(1, n_dir) * 6);
    if (!dd || !de) return fail(h, MOT_EOOM, "device allocation (far field)");
    CK(cudaMemcpy(dd, dirs, sizeof(double) * 3 * n_dir, cudaMemcpyHostToDevice));
    CK(cudaStreamWaitEvent(0, h->ev_state, 0));  // the Fourier sums of the last step, on whatever stream it ran
    launch_far_field(h, n_dir, dd, de, 0);
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(E_out, de, sizeof(double) * (size_t)h->B * h->nfreq * n_dir * 6, cudaMemcpyDeviceToHost));
    cudaFree(dd);
    cudaFree(de);
    h->device_bytes -= (int64_t)(sizeof(double) * 3 * std::max(1, n_dir) +
                                 sizeof(double) * (size_t)h->B * h->nfreq * std::max(1, n_dir) * 6);
    return MOT_OK;
}

MOT_API int mot_reset(mot_handle* h) {
    if (!h) return MOT_EINVAL;
    CK(cudaSetDevice(h->dev));
    CK(cudaDeviceSynchronize());
    free_state(h);
    return MOT_OK;
}

namespace {
struct StateHeader {
    uint64_t magic;
    int32_t ne, B, R, nfreq, npad, pad;
    int64_t step;
};
const uint64_t kMagic = 0x4d4f545354415430ULL;
}  // namespace

MOT_API int mot_save_state(mot_handle* h, void* buf, size_t* size) {
    if (!h || !size) return MOT_EINVAL;
    if (!h->d_ring) return fail(h, MOT_ESTATE, "no march state");
    const size_t bv = (size_t)h->npad * 2 * h->B;
    const size_t ring = sizeof(double) * (size_t)h->R * 6 * bv;
    const size_t cur = sizeof(double) * 4 * (size_t)h->npad * h->B;
    const size_t dft = sizeof(double) * std::max(1, h->nfreq) * 4 * (size_t)h->npad * h->B * 2;
    const size_t wp = sizeof(double) * bv;
    const size_t need = sizeof(StateHeader) + sizeof(double) * 10 * h->B + ring + cur + dft + 2 * wp;
    if (!buf) {
        *size = need;
        return MOT_OK;
    }
    if (*size < need) return fail(h, MOT_EINVAL, "state buffer too small");
    CK(cudaSetDevice(h->dev));
    CK(cudaDeviceSynchronize());
    StateHeader hd{kMagic, h->ne, h->B, h->R, h->nfreq, h->npad, 0, h->step};
    char* p = (char*)buf;
    memcpy(p, &hd, sizeof hd);
    p += sizeof hd;
    memcpy(p, h->h_waves.data(), sizeof(double) * 10 * h->B);
    p += sizeof(double) * 10 * h->B;
    CK(cudaMemcpy(p, h->d_ring, ring, cudaMemcpyDeviceToHost));
    p += ring;
    CK(cudaMemcpy(p, h->d_cur, cur, cudaMemcpyDeviceToHost));
    p += cur;
    CK(cudaMemcpy(p, h->d_dft, dft, cudaMemcpyDeviceToHost));
    p += dft;
    CK(cudaMemcpy(p, h->d_wprev1, wp, cudaMemcpyDeviceToHost));
    p += wp;
    CK(cudaMemcpy(p, h->d_wprev2, wp, cudaMemcpyDeviceToHost));
    *size = need;
    return MOT_OK;
}

MOT_API int mot_load_state(mot_handle* h, const void* buf, size_t size) {
    if (!h || !buf) return MOT_EINVAL;
    if (!h->loaded) return fail(h, MOT_ESTATE, "load operators first");
    StateHeader hd;
    if (size < sizeof hd) return fail(h, MOT_EINVAL, "state buffer too small");
    memcpy(&hd, buf, sizeof hd);
    if (hd.magic != kMagic || hd.ne != h->ne || hd.R != h->R || hd.npad != h->npad || hd.nfreq != h->nfreq ||
        hd.B < 1 || hd.B > MOT_MAX_B)
        return fail(h, MOT_EINVAL, "state does not match this handle");
    CK(cudaSetDevice(h->dev));
    if (h->B != hd.B) {
        free_state(h);
    }
    int st;
    if ((st = ensure_state(h, hd.B)) != MOT_OK) return st;
    const size_t bv = (size_t)h->npad * 2 * h->B;
    const size_t ring = sizeof(double) * (size_t)h->R * 6 * bv;
    const size_t cur = sizeof(double) * 4 * (size_t)h->npad * h->B;
    const size_t dft = sizeof(double) * std::max(1, h->nfreq) * 4 * (size_t)h->npad * h->B * 2;
    const size_t wp = sizeof(double) * bv;
    if (size < sizeof hd + sizeof(double) * 10 * h->B + ring + cur + dft + 2 * wp)
        return fail(h, MOT_EINVAL, "state buffer too small");
    const char* p = (const char*)buf + sizeof hd;
    h->h_waves.assign((const double*)p, (const double*)p + 10 * h->B);
    CK(cudaMemcpy(h->d_waves, p, sizeof(double) * 10 * h->B, cudaMemcpyHostToDevice));
    p += sizeof(double) * 10 * h->B;
    CK(cudaMemcpy(h->d_ring, p, ring, cudaMemcpyHostToDevice));
    p += ring;
    CK(cudaMemcpy(h->d_cur, p, cur, cudaMemcpyHostToDevice));
    p += cur;
    CK(cudaMemcpy(h->d_dft, p, dft, cudaMemcpyHostToDevice));
    p += dft;
    CK(cudaMemcpy(h->d_wprev1, p, wp, cudaMemcpyHostToDevice));
    p += wp;
    CK(cudaMemcpy(h->d_wprev2, p, wp, cudaMemcpyHostToDevice));
    // reduced-precision copies of the ring used by the mixed history kernels
    if (h->hist_tc)
        for (int slot = 0; slot < h->R; slot++) launch_split_ring(h, slot, 0);
    else if (h->d_ring32)
        launch_d2f(h, (size_t)h->R * 6 * bv, h->d_ring, h->d_ring32, 0);
    CK(cudaDeviceSynchronize());
    h->step = hd.step;
    return MOT_OK;
}

MOT_API int mot_get_info(mot_handle* h, mot_info* info) {
    if (!h || !info) return MOT_EINVAL;
    info->ne = h->ne;
    info->nv = h->nv;
    info->nf = h->nf;
    info->kmax = h->kmax;
    info->K = h->K;
    info->B = h->B;
    info->step = h->step;
    info->D = h->D;
    info->tmax = h->tmax;
    info->dt = h->dt;
    info->last_gmres_iters = h->last_gmres_iters;
    info->last_gmres_resid = h->last_gmres_resid;
    info->last_cg_iters = h->last_cg_iters;
    info->device_bytes = h->device_bytes;
    info->gpu_launches = h->launches;
    info->tile_fill = h->tile_fill;
    info->tile_count = h->ntiles;
    const double Bc = std::max(1, h->B);
    info->hist_flops_per_step = 2.0 * h->hist_nnz_tasks * 2.0 * Bc;
    // values at the precision the path stores them: FP64, or FP32 on the mixed path
    const double vb = h->opt.precision == MOT_PREC_MIXED ? 4.0 : 8.0;
    info->hist_bytes_per_step = vb * h->hist_nnz_unique + vb * (double)h->K * 2.0 * 2.0 * h->ne * Bc;
    info->hist_tc_tasks = h->hist_tc_list.ntasks;
    info->gmres_iters_total = h->gmres_iters_total;
    info->tc_chunk_cap = h->tc_cap;
    info->tc_lag_frac = h->tc_lag_frac;
    info->tc_stages = h->tc_stages;
    info->tc_epilogue_warps = h->tc_epi;
    info->tc_tasks_per_stage = h->tc_tps;
    info->tc_tuned = h->tc_tuned ? 1 : 0;
    info->tc_tune_ms = h->tc_tune_ms;
    info->tc_launches = h->tc_launches;
    info->hist_timed_launches = h->timed_launches;
    info->hist_timed_ms = h->timed_ms;
    for (int k = 0; k < 8; k++) info->phase_ms[k] = h->phase_ms[k];
    info->hist_kernel = h->hist_tc ? 2 : (h->opt.precision == MOT_PREC_MIXED && mflag(h, MOT_MIX_HIST32)) ? 1 : 0;
    return MOT_OK;
}

MOT_API int mot_get_edges(mot_handle* h, int32_t* ev, int32_t* ef) {
    if (!h || !ev || !ef) return MOT_EINVAL;
    memcpy(ev, h->ev.data(), sizeof(int) * 2 * h->ne);
    memcpy(ef, h->ef.data(), sizeof(int) * 2 * h->ne);
    return MOT_OK;
}

MOT_API const char* mot_last_error(mot_handle* h) { return h ? h->err.c_str() : "null handle"; }

MOT_API void mot_destroy(mot_handle* h) {
    if (!h) return;
    cudaSetDevice(h->dev);
    cudaDeviceSynchronize();
    free_state(h);
    void* ptrs[] = {h->d_edge_faces, h->d_edge_verts, h->d_face_edges, h->d_face_sgn, h->d_iperm, h->d_cg_iters,
                    h->vtx_edges.rowptr, h->vtx_edges.col, h->vtx_edges.val, h->Lf.rowptr, h->Lf.col, h->Lf.val,
                    h->Lv.rowptr, h->Lv.col, h->Lv.val, h->G.rowptr, h->G.col, h->G.val, h->Gt.rowptr,
                    h->Gt.col, h->Gt.val, h->d_T0s, h->d_T0h, h->d_rhs_x, h->d_rhs_wf, h->d_tiles,
                    h->hist.tasks, h->hist.chunks, h->hist.chunk_ptr, h->lag0.tasks, h->lag0.chunks,
                    h->lag0.chunk_ptr, h->d_omega, h->d_colidx, h->d_tiles32, h->d_Q0, h->d_Q0f, h->d_LF,
                    h->d_LFf, h->d_Minvf, h->d_Minv64, h->d_Lfinvf, h->hist_tc_list.packed, h->hist_tc_list.chunks,
                    h->hist_tc_list.rb_ptr, h->hist_tc_list.rb_chunks, h->d_tiles16, h->d_sgws, h->d_emuws,
                    h->d_Ginv64, h->d_Lfinv64, h->d_Lvinv64, h->d_dir_r, h->d_dir_z, h->d_dir_sc};
    emu_free(h, &h->emu_Q0);
    emu_free(h, &h->emu_LF);
    emu_free(h, &h->emu_Q0s);
    emu_free(h, &h->emu_Minv);
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (h->h_cg_iters) cudaFreeHost(h->h_cg_iters);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->ev_state) cudaEventDestroy(h->ev_state);
    for (int k = 0; k < 8; k++)
        if (h->pev[k]) cudaEventDestroy(h->pev[k]);
    delete h;
}
