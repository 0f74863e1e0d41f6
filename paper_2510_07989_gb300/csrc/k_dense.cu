// Dense FP64 factorisation used once at load time by the mixed path: blocked
// right-looking LU with partial pivoting of the dense Q_0 and its explicit
// inverse (the GMRES preconditioner M ~ Q_0^{-1}, applied in FP32).
//
// All matrices are row-major n x n with leading dimension n (n a multiple of
// the block size 64).
#include <math.h>

#include "mot_internal.h"

namespace {

constexpr int NB = 64;

// argmax_{r >= j} |A[r][j]| -> piv[j]; one CTA.
__global__ void k_pivot(int n, double* __restrict__ A, int j, int* __restrict__ piv) {
    __shared__ double bv[1024];
    __shared__ int bi[1024];
    double best = -1.0;
    int bidx = j;
    for (int r = j + threadIdx.x; r < n; r += blockDim.x) {
        const double v = fabs(A[(size_t)r * n + j]);
        if (v > best) {
            best = v;
            bidx = r;
        }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = bidx;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            const double o = bv[threadIdx.x + st];
            const int oi = bi[threadIdx.x + st];
            if (o > bv[threadIdx.x] || (o == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
                bv[threadIdx.x] = o;
                bi[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) piv[j] = bi[0];
}

// swap rows j and piv[j] over all n columns
__global__ void k_swap(int n, double* __restrict__ A, int j, const int* __restrict__ piv) {
    const int p = piv[j];
    if (p == j) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const double t = A[(size_t)j * n + c];
        A[(size_t)j * n + c] = A[(size_t)p * n + c];
        A[(size_t)p * n + c] = t;
    }
}

// rows r > j: l = A[r][j] / A[j][j] stored in place; A[r][c] -= l A[j][c] for c in (j, jend)
__global__ void k_panel_update(int n, double* __restrict__ A, int j, int jend) {
    const double d = A[(size_t)j * n + j];
    for (int r = j + 1 + blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        double* row = A + (size_t)r * n;
        const double l = d != 0.0 ? row[j] / d : 0.0;
        row[j] = l;
        const double* pr = A + (size_t)j * n;
        for (int c = j + 1; c < jend; c++) row[c] -= l * pr[c];
    }
}

// X[k0..k0+NB)[c] <- L11^{-1} X[...][c] for columns c in [c0, n) (unit lower L11 = A block)
__global__ void k_trsm_lower_unit(int n, const double* __restrict__ A, int k0, double* __restrict__ X, int ldx,
                                  int c0, int ncol) {
    for (int c = c0 + blockIdx.x * blockDim.x + threadIdx.x; c < c0 + ncol; c += gridDim.x * blockDim.x) {
        double y[NB];
        for (int i = 0; i < NB; i++) {
            double v = X[(size_t)(k0 + i) * ldx + c];
            for (int q = 0; q < i; q++) v -= A[(size_t)(k0 + i) * n + k0 + q] * y[q];
            y[i] = v;
        }
        for (int i = 0; i < NB; i++) X[(size_t)(k0 + i) * ldx + c] = y[i];
    }
}

// X[k0..k0+NB)[c] <- U11^{-1} X[...][c] (upper, non-unit diagonal)
__global__ void k_trsm_upper(int n, const double* __restrict__ A, int k0, double* __restrict__ X, int ldx, int c0,
                             int ncol) {
    for (int c = c0 + blockIdx.x * blockDim.x + threadIdx.x; c < c0 + ncol; c += gridDim.x * blockDim.x) {
        double y[NB];
        for (int i = NB - 1; i >= 0; i--) {
            double v = X[(size_t)(k0 + i) * ldx + c];
            for (int q = i + 1; q < NB; q++) v -= A[(size_t)(k0 + i) * n + k0 + q] * y[q];
            const double dg = A[(size_t)(k0 + i) * n + k0 + i];
            y[i] = dg != 0.0 ? v / dg : 0.0;
        }
        for (int i = 0; i < NB; i++) X[(size_t)(k0 + i) * ldx + c] = y[i];
    }
}

// C[M][N] -= A[M][K] B[K][N] (strided), FP64, 64 x 64 tiles, 4 x 4 per thread.
constexpr int DT = 64, DK = 16;
__global__ void __launch_bounds__(256) k_dgemm_sub(int M, int N, int K, const double* __restrict__ A, int lda,
                                                   const double* __restrict__ B, int ldb, double* __restrict__ C,
                                                   int ldc) {
    __shared__ double sa[DK][DT + 1];
    __shared__ double sb[DK][DT];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int r0 = blockIdx.y * DT, c0 = blockIdx.x * DT;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < K; k0 += DK) {
        for (int e = threadIdx.x; e < DT * DK; e += 256) {
            const int r = e / DK, k = e - r * DK;
            sa[k][r] = (r0 + r < M && k0 + k < K) ? A[(size_t)(r0 + r) * lda + k0 + k] : 0.0;
        }
        for (int e = threadIdx.x; e < DK * DT; e += 256) {
            const int k = e / DT, c = e - k * DT;
            sb[k][c] = (k0 + k < K && c0 + c < N) ? B[(size_t)(k0 + k) * ldb + c0 + c] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < DK; k++) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = sa[k][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = sb[k][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int r = r0 + ty * 4 + i;
        if (r >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int c = c0 + tx * 4 + j;
            if (c < N) C[(size_t)r * ldc + c] -= acc[i][j];
        }
    }
}

// X = P (permutation of the identity by the recorded row swaps, applied in order)
__global__ void k_identity(int n, double* __restrict__ X) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)n * n; i += (size_t)gridDim.x * blockDim.x)
        X[i] = (i / n == i % n) ? 1.0 : 0.0;
}

__global__ void k_count_bad(int n, const double* __restrict__ A, int* __restrict__ bad) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (!(fabs(A[(size_t)i * n + i]) > 0.0) || !isfinite(A[(size_t)i * n + i])) atomicAdd(bad, 1);
}

// unit diagonal on the padded (edge >= ne) rows/columns of an interleaved (2 npad)^2 operator
__global__ void k_pad_identity(int n, int ne, double* __restrict__ A) {
    for (int J = 2 * ne + blockIdx.x * blockDim.x + threadIdx.x; J < n; J += gridDim.x * blockDim.x)
        A[(size_t)J * n + J] = 1.0;
}

// A (npd x npd) = L + (1/n) 1 1^T on the leading n x n block (L in CSR), identity on the padding
__global__ void k_lap_plus_j(int n, int npd, const int* __restrict__ rp, const int* __restrict__ ci,
                             const double* __restrict__ va, double* __restrict__ A) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)npd * npd;
         e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / npd), j = (int)(e % npd);
        A[e] = (i < n && j < n) ? 1.0 / n : (i == j ? 1.0 : 0.0);
    }
}
__global__ void k_lap_add_csr(int n, int npd, const int* __restrict__ rp, const int* __restrict__ ci,
                              const double* __restrict__ va, double* __restrict__ A) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int j = rp[i]; j < rp[i + 1]; j++) A[(size_t)i * npd + ci[j]] += va[j];
}

// per-column dot products of two N x C row-major blocks: partial[chunk][c]
__global__ void k_coldot(int N, int C, const double* __restrict__ X, const double* __restrict__ Y,
                         double* __restrict__ partial) {
    const int c = threadIdx.x % C, rs = threadIdx.x / C, RS = blockDim.x / C;
    double s = 0.0;
    if (threadIdx.x < RS * C)
        for (int r = blockIdx.x * 64 + rs; r < min(N, blockIdx.x * 64 + 64); r += RS)
            s = fma(X[(size_t)r * C + c], Y[(size_t)r * C + c], s);
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < C) {
        double t = 0.0;
        for (int k = 0; k < RS; k++) t += red[k * C + threadIdx.x];
        partial[(size_t)blockIdx.x * C + threadIdx.x] = t;
    }
}
__global__ void k_coldot_reduce(int nchunk, int C, const double* __restrict__ partial, double* __restrict__ out) {
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < nchunk; k++) s += partial[(size_t)k * C + c];
        out[c] = s;
    }
}
// r[row][c] = f[row][c] - mean over the N rows of column c (one CTA per column):
// the consistent part of a graph-Laplacian right-hand side (see pcg_dense_prec)
// It is also scaled by a power of two to O(1) (exact); unscale[c] receives
// the inverse factor, which the solution is multiplied by at the end.
__global__ void k_demean_cols(int N, int C, const double* __restrict__ f, double* __restrict__ r,
                              double* __restrict__ unscale) {
    __shared__ double red[256];
    const int c = blockIdx.x;
    double s = 0.0;
    for (int row = threadIdx.x; row < N; row += blockDim.x) s += f[(size_t)row * C + c];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const double mean = red[0] / (double)N;
    __syncthreads();
    double m = 0.0;
    for (int row = threadIdx.x; row < N; row += blockDim.x) m = fmax(m, fabs(f[(size_t)row * C + c] - mean));
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    const int e = red[0] > 0.0 ? ilogb(red[0]) : 0;
    const double sc = ldexp(1.0, -e);
    for (int row = threadIdx.x; row < N; row += blockDim.x)
        r[(size_t)row * C + c] = (f[(size_t)row * C + c] - mean) * sc;
    if (threadIdx.x == 0) unscale[c] = ldexp(1.0, e);
}
// z[row][c] *= f[c]
__global__ void k_scale_cols(int N, int C, const double* __restrict__ f, double* __restrict__ z) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)N * C;
         e += (size_t)gridDim.x * blockDim.x)
        z[e] *= f[e % C];
}
// x += a p ; r -= a q with a = num/den per column (0 if den <= 0 or the column is done)
__global__ void k_pcg_xr(int N, int C, const double* __restrict__ num, const double* __restrict__ den,
                         const int* __restrict__ done, const double* __restrict__ p, const double* __restrict__ q,
                         double* __restrict__ x, double* __restrict__ r) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)N * C;
         e += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        const double a = (!done[c] && den[c] > 0.0) ? num[c] / den[c] : 0.0;
        x[e] += a * p[e];
        r[e] -= a * q[e];
    }
}
// p = z + (num/den) p per column
__global__ void k_pcg_p(int N, int C, const double* __restrict__ num, const double* __restrict__ den,
                        const double* __restrict__ z, double* __restrict__ p) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)N * C;
         e += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        const double b = den[c] > 0.0 ? num[c] / den[c] : 0.0;
        p[e] = z[e] + b * p[e];
    }
}

inline void dgemm_sub(mot_handle* h, int M, int N, int K, const double* A, int lda, const double* B, int ldb,
                      double* C, int ldc, cudaStream_t s) {
    if (M <= 0 || N <= 0 || K <= 0) return;
    dim3 grid((N + DT - 1) / DT, (M + DT - 1) / DT);
    k_dgemm_sub<<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc);
    h->launches++;
}

}  // namespace

namespace mot {

void launch_sgemm_d(mot_handle* h, int M, int N, int K, const float* A, const float* X, double* Y, cudaStream_t s);
void launch_d2f(mot_handle* h, size_t n, const double* x, float* y, cudaStream_t s);

void dense_lap_plus_j(mot_handle* h, const DCsr& L, int npd, double* A, cudaStream_t s) {
    k_lap_plus_j<<<1024, 256, 0, s>>>(L.n, npd, L.rowptr, L.col, L.val, A);
    k_lap_add_csr<<<(L.n + 255) / 256, 256, 0, s>>>(L.n, npd, L.rowptr, L.col, L.val, A);
    h->launches += 2;
}

// Preconditioned FP64 CG on a graph Laplacian L (CSR, N rows) for C columns:
// L z = f with f orthogonal to the constants up to rounding (its column mean
// is removed first), M an FP32 copy of (L + 11^T/N)^{-1}
// (npd x npd, npd >= N, zero padded rows). work: 5 blocks of npd x C doubles,
// d_scal: 6*C doubles + C ints, fstage: npd*C floats. Returns iterations (or -1).
int pcg_dense_prec(mot_handle* h, const DCsr& L, int npd, const float* M, const double* f, int C, double* z,
                   double* work, double* d_scal, float* fstage, double tol, int maxit, cudaStream_t s) {
    const int N = L.n;
    const size_t blk = (size_t)npd * C;
    double* r = work;
    double* p = r + blk;
    double* q = p + blk;
    double* zz = q + blk;
    double* red = zz + blk;  // partials: ceil(npd/64) * C
    double* rz = d_scal;
    double* rzn = rz + C;
    double* pq = rzn + C;
    double* rr = pq + C;
    double* ff = rr + C;
    int* done = (int*)(ff + C);
    double* unscale = ff + 2 * C;  // after the C ints of done (room for C doubles)
    const int nch = (N + 63) / 64;
    auto coldot = [&](const double* X, const double* Y, double* out) {
        k_coldot<<<nch, 256, 0, s>>>(N, C, X, Y, red);
        k_coldot_reduce<<<1, 256, 0, s>>>(nch, C, red, out);
        h->launches += 2;
    };
    auto precond = [&](const double* in, double* out) {  // out = M in (rows npd, FP32 products, FP64 sums)
        launch_d2f(h, blk, in, fstage, s);
        launch_sgemm_d(h, npd, C, npd, M, fstage, out, s);
    };
    const int g = (int)std::min<size_t>(4096, (blk + 255) / 256);
    cudaMemsetAsync(z, 0, sizeof(double) * blk, s);
    cudaMemsetAsync(done, 0, sizeof(int) * C, s);
    cudaMemsetAsync(r, 0, sizeof(double) * blk, s);  // padded rows must be zero (finite) for M
    // f sums to zero only up to rounding; its mean is an inconsistent part that
    // CG cannot reduce, sizeable when x lies almost entirely in the loop space
    k_demean_cols<<<C, 256, 0, s>>>(N, C, f, r, unscale);
    h->launches++;
    coldot(r, r, ff);
    precond(r, zz);
    cudaMemcpyAsync(p, zz, sizeof(double) * blk, cudaMemcpyDeviceToDevice, s);
    coldot(r, zz, rz);
    std::vector<double> hr(C), hf(C);
    std::vector<int> hd(C, 0);
    cudaMemcpyAsync(hf.data(), ff, sizeof(double) * C, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    int it = 0;
    for (; it < maxit; it++) {
        // q = L p
        launch_spmv(h, L, p, C, q, s);
        coldot(p, q, pq);
        k_pcg_xr<<<g, 256, 0, s>>>(N, C, rz, pq, done, p, q, z, r);
        coldot(r, r, rr);
        cudaMemcpyAsync(hr.data(), rr, sizeof(double) * C, cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        h->launches++;
        bool all = true;
        for (int c = 0; c < C; c++) {
            if (!hd[c] && !(hr[c] > tol * tol * hf[c])) hd[c] = 1;
            all &= hd[c] != 0;
        }
        if (all) {
            it++;
            break;
        }
        cudaMemcpyAsync(done, hd.data(), sizeof(int) * C, cudaMemcpyHostToDevice, s);
        precond(r, zz);
        coldot(r, zz, rzn);
        k_pcg_p<<<g, 256, 0, s>>>(N, C, rzn, rz, zz, p);
        cudaMemcpyAsync(rz, rzn, sizeof(double) * C, cudaMemcpyDeviceToDevice, s);
        h->launches++;
    }
    k_scale_cols<<<g, 256, 0, s>>>(N, C, unscale, z);
    h->launches++;
    return it;
}

// Direct solve of a graph-Laplacian system L z = f (N rows, C columns), the
// consistent one: the column mean of f is removed (and the column scaled by a
// power of two, undone at the end), then z = Linv r with Linv the dense FP64
// (L + 11^T/N)^{-1} (npd x npd, identity on the padding), which on mean-free
// right-hand sides is the pseudo-inverse (minimum-norm solution).
// r, z: npd x C doubles each; sc: C doubles.
void direct_laplacian_solve(mot_handle* h, int N, int npd, const double* Linv, const double* f, int C, double* r,
                            double* z, double* sc, cudaStream_t s) {
    cudaMemsetAsync(r, 0, sizeof(double) * (size_t)npd * C, s);  // padded rows: zero
    k_demean_cols<<<C, 256, 0, s>>>(N, C, f, r, sc);
    h->launches++;
    launch_gemm_rect(h, npd, npd, Linv, r, C, z, s);
    const size_t blk = (size_t)N * C;
    k_scale_cols<<<(int)std::min<size_t>(4096, (blk + 255) / 256), 256, 0, s>>>(N, C, sc, z);
    h->launches++;
}

void dense_pad_identity(mot_handle* h, int n, int ne, double* A, cudaStream_t s) {
    if (2 * ne >= n) return;
    k_pad_identity<<<(n - 2 * ne + 255) / 256, 256, 0, s>>>(n, ne, A);
    h->launches++;
}

// In place LU (P A = L U) of the n x n matrix A; piv (device, n ints) records the swaps.
// Returns the number of zero or non-finite pivots (0 on success).
int dense_lu(mot_handle* h, int n, double* A, int* piv, int* d_bad, cudaStream_t s) {
    for (int k0 = 0; k0 < n; k0 += NB) {
        const int k1 = k0 + NB;
        for (int j = k0; j < k1; j++) {
            k_pivot<<<1, 1024, 0, s>>>(n, A, j, piv);
            k_swap<<<(n + 255) / 256, 256, 0, s>>>(n, A, j, piv);
            k_panel_update<<<(n - j + 255) / 256 + 1, 256, 0, s>>>(n, A, j, k1);
            h->launches += 3;
        }
        if (k1 < n) {
            k_trsm_lower_unit<<<(n - k1 + 127) / 128, 128, 0, s>>>(n, A, k0, A, n, k1, n - k1);
            dgemm_sub(h, n - k1, n - k1, NB, A + (size_t)k1 * n + k0, n, A + (size_t)k0 * n + k1, n,
                      A + (size_t)k1 * n + k1, n, s);
            h->launches++;
        }
    }
    cudaMemsetAsync(d_bad, 0, sizeof(int), s);
    k_count_bad<<<(n + 255) / 256, 256, 0, s>>>(n, A, d_bad);
    h->launches++;
    int bad = 0;
    cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    return bad;
}

// X = A^{-1} from the LU factors: X = U^{-1} L^{-1} P, blocked right-looking solves.
void dense_inverse_from_lu(mot_handle* h, int n, const double* LU, const int* piv, double* X, cudaStream_t s) {
    k_identity<<<1024, 256, 0, s>>>(n, X);
    h->launches++;
    for (int j = 0; j < n; j++) {  // apply the recorded swaps to the identity
        k_swap<<<(n + 255) / 256, 256, 0, s>>>(n, X, j, piv);
        h->launches++;
    }
    for (int k0 = 0; k0 < n; k0 += NB) {  // L Y = P X
        const int k1 = k0 + NB;
        k_trsm_lower_unit<<<(n + 127) / 128, 128, 0, s>>>(n, LU, k0, X, n, 0, n);
        dgemm_sub(h, n - k1, n, NB, LU + (size_t)k1 * n + k0, n, X + (size_t)k0 * n, n, X + (size_t)k1 * n, n, s);
        h->launches++;
    }
    for (int k0 = n - NB; k0 >= 0; k0 -= NB) {  // U X = Y
        k_trsm_upper<<<(n + 127) / 128, 128, 0, s>>>(n, LU, k0, X, n, 0, n);
        dgemm_sub(h, k0, n, NB, LU + k0, n, X + (size_t)k0 * n, n, X, n, s);
        h->launches++;
    }
}

}  // namespace mot
