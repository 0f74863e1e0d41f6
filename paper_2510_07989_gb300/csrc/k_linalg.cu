// Kernels of the MOT step other than the history contraction: incidence
// products and FP64 CG solves behind the quasi-Helmholtz projectors
// (paper Section IV-B), the Gram solve and the static preconditioner products
// (Section III, Eq. (CP)), the right-hand side (Section V-C), current recovery
// and running Fourier sums (Eq. (dis_jm)), and the batched GMRES pieces of the
// Q_0 solve (Eq. (MOT)).
//
// Block vectors are row-major [rows][C]: row = edge (or face / vertex),
// column = one right-hand side component (u-part columns 0..B-1, v-part B..2B-1).
#include <math.h>

#include "mot_internal.h"

namespace {

// ----------------------------------------------------------------- helpers
__global__ void k_axpby(int n, double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                        double* __restrict__ z) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double v = a * x[i];
        if (y) v += b * y[i];
        z[i] = v;
    }
}

// dst[v][npad][C2]: v=0: [eta u, v/eta], v=1: [eta' u, v/eta'], v=2: [-v, u]
__global__ void k_variants(int npad, int B, const double* __restrict__ x, double* __restrict__ dst, double eta,
                           double etap) {
    const int C2 = 2 * B;
    const size_t ps = (size_t)npad * C2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npad * B; i += gridDim.x * blockDim.x) {
        const int r = i / B, b = i - r * B;
        const double u = x[(size_t)r * C2 + b], v = x[(size_t)r * C2 + B + b];
        dst[(size_t)r * C2 + b] = eta * u;
        dst[(size_t)r * C2 + B + b] = v / eta;
        dst[ps + (size_t)r * C2 + b] = etap * u;
        dst[ps + (size_t)r * C2 + B + b] = v / etap;
        dst[2 * ps + (size_t)r * C2 + b] = -v;
        dst[2 * ps + (size_t)r * C2 + B + b] = u;
    }
}

// f[face][c] = sum over the face's edges of Sigma_{e,face} x[e][c]   (Sigma^T x)
__global__ void k_sigma_t(int nf, int C, const int* __restrict__ fe, const double* __restrict__ fs,
                          const double* __restrict__ x, double* __restrict__ f) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nf * C; i += gridDim.x * blockDim.x) {
        const int r = i / C, c = i - r * C;
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < 3; j++) s += fs[3 * r + j] * x[(size_t)fe[3 * r + j] * C + c];
        f[i] = s;
    }
}

// x[e][c] = z[c+(e)][c] - z[c-(e)][c]   (Sigma z)
__global__ void k_sigma(int ne, int C, const int* __restrict__ ef, const double* __restrict__ z,
                        double* __restrict__ x) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ne * C; i += gridDim.x * blockDim.x) {
        const int r = i / C, c = i - r * C;
        x[i] = z[(size_t)ef[2 * r] * C + c] - z[(size_t)ef[2 * r + 1] * C + c];
    }
}

// x[e][c] = z[v+(e)][c] - z[v-(e)][c]   (Lambda z)
__global__ void k_lambda(int ne, int C, const int* __restrict__ ev, const double* __restrict__ z,
                         double* __restrict__ x) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ne * C; i += gridDim.x * blockDim.x) {
        const int r = i / C, c = i - r * C;
        x[i] = z[(size_t)ev[2 * r + 1] * C + c] - z[(size_t)ev[2 * r] * C + c];
    }
}

// y = A x for a CSR matrix (rows A.n), C columns
__global__ void k_spmv(int n, int C, const int* __restrict__ rp, const int* __restrict__ ci,
                       const double* __restrict__ va, const double* __restrict__ x, double* __restrict__ y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * C; i += gridDim.x * blockDim.x) {
        const int r = i / C, c = i - r * C;
        double s = 0.0;
        for (int j = rp[r]; j < rp[r + 1]; j++) s = fma(va[j], x[(size_t)ci[j] * C + c], s);
        y[i] = s;
    }
}

// ----------------------------------------------------------------- CG
// Solves A z = f column by column (A SPD, or singular and consistent: the
// Laplacians Sigma^T Sigma and Lambda^T Lambda, whose null space is the
// constants; f = Sigma^T x / Lambda^T x is orthogonal to it up to rounding,
// and its column mean is removed before the iteration). With NORMAL the
// operator is A2 (A x) (CGNR for the Gram matrix: A = G, A2 = G^T).
// One CTA owns CW columns (lane % CW) and all rows; only __syncthreads is used.
struct CsrV {
    const int* rp;
    const int* ci;
    const double* va;
};

template <int CW>
__device__ __forceinline__ double col_reduce(double v, double* red, double* colv) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off >= CW; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane < CW) red[warp * CW + lane] = v;
    __syncthreads();
    if (threadIdx.x < CW) {
        double s = 0.0;
        const int nw = blockDim.x >> 5;
        for (int w = 0; w < nw; w++) s += red[w * CW + threadIdx.x];
        colv[threadIdx.x] = s;
    }
    __syncthreads();
    const double r = colv[lane % CW];
    __syncthreads();
    return r;
}

template <int CW>
__device__ __forceinline__ double col_reduce_max(double v, double* red, double* colv) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off >= CW; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    if (lane < CW) red[warp * CW + lane] = v;
    __syncthreads();
    if (threadIdx.x < CW) {
        double m = 0.0;
        const int nw = blockDim.x >> 5;
        for (int w = 0; w < nw; w++) m = fmax(m, red[w * CW + threadIdx.x]);
        colv[threadIdx.x] = m;
    }
    __syncthreads();
    const double r = colv[lane % CW];
    __syncthreads();
    return r;
}

// 2^-e with 2^e the power of two at or below m (1 for m = 0): multiplying by
// it (and later by its inverse) is exact and brings a column to O(1)
__device__ __forceinline__ double pow2_scale(double m) { return m > 0.0 ? ldexp(1.0, -ilogb(m)) : 1.0; }

template <int CW, bool NORMAL>
__global__ void __launch_bounds__(1024) k_cg(int N, int C, CsrV A, CsrV A2, const double* __restrict__ f,
                                             double* __restrict__ z, double* __restrict__ r, double* __restrict__ p,
                                             double* __restrict__ q, double* __restrict__ t, double tol, int maxit,
                                             int* __restrict__ it_max, int* __restrict__ noconv) {
    __shared__ double red[32 * CW];
    __shared__ double colv[CW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cl = lane % CW;
    const int c = blockIdx.x * CW + cl;
    const bool cv = c < C;
    const int RPW = 32 / CW;
    const int row0 = warp * RPW + lane / CW;
    const int RS = (blockDim.x >> 5) * RPW;
    double part = 0.0;
    // A graph Laplacian (not NORMAL) is singular with the constants as its null
    // space (connected surface). Its right-hand sides (Sigma^T x, Lambda^T x) sum
    // to zero only up to rounding; when x lies almost entirely in the other
    // subspace, that rounding is a sizeable inconsistent part of f, which CG
    // cannot reduce (the iteration then runs to its limit and drifts along the
    // null space). The column mean is removed first, so the solve is the
    // consistent one whose minimum-norm solution is the pseudo-inverse of
    // Section IV-B applied to f.
    double mean = 0.0;
    if (!NORMAL) {
        for (int row = row0; row < N; row += RS)
            if (cv) part += f[(size_t)row * C + c];
        mean = col_reduce<CW>(part, red, colv) / (double)N;
        part = 0.0;
    }
    // the column is scaled by a power of two to O(1) (exact) and the solution
    // scaled back at the end, so sums of squares neither underflow nor
    // overflow whatever the scale of f (late in a march f decays without bound)
    for (int row = row0; row < N; row += RS)
        if (cv) part = fmax(part, fabs(f[(size_t)row * C + c] - mean));
    const double sc = pow2_scale(col_reduce_max<CW>(part, red, colv));
    part = 0.0;
    for (int row = row0; row < N; row += RS)
        if (cv) {
            const size_t ix = (size_t)row * C + c;
            const double v = (f[ix] - mean) * sc;
            z[ix] = 0.0;
            r[ix] = v;
            p[ix] = v;
            part += v * v;
        }
    double rr = col_reduce<CW>(part, red, colv);
    const double bb = rr;
    bool done = !(bb > 0.0) || !cv;
    int it = 0;
    while (it < maxit) {
        if (__syncthreads_and(done)) break;
        if (NORMAL) {
            for (int row = row0; row < N; row += RS)
                if (cv) {
                    double s = 0.0;
                    for (int j = A.rp[row]; j < A.rp[row + 1]; j++) s = fma(A.va[j], p[(size_t)A.ci[j] * C + c], s);
                    t[(size_t)row * C + c] = s;
                }
            __syncthreads();
        }
        part = 0.0;
        for (int row = row0; row < N; row += RS)
            if (cv) {
                double s = 0.0;
                if (NORMAL) {
                    for (int j = A2.rp[row]; j < A2.rp[row + 1]; j++)
                        s = fma(A2.va[j], t[(size_t)A2.ci[j] * C + c], s);
                } else {
                    for (int j = A.rp[row]; j < A.rp[row + 1]; j++) s = fma(A.va[j], p[(size_t)A.ci[j] * C + c], s);
                }
                q[(size_t)row * C + c] = s;
                part += p[(size_t)row * C + c] * s;
            }
        const double pq = col_reduce<CW>(part, red, colv);
        const double alpha = (done || !(pq > 0.0)) ? 0.0 : rr / pq;
        part = 0.0;
        for (int row = row0; row < N; row += RS)
            if (cv) {
                const size_t ix = (size_t)row * C + c;
                z[ix] += alpha * p[ix];
                const double rv = r[ix] - alpha * q[ix];
                r[ix] = rv;
                part += rv * rv;
            }
        const double rn = col_reduce<CW>(part, red, colv);
        const double beta = done ? 0.0 : rn / rr;
        if (!done) {
            rr = rn;
            if (rr <= tol * tol * bb) done = true;
        }
        for (int row = row0; row < N; row += RS)
            if (cv && !done) {
                const size_t ix = (size_t)row * C + c;
                p[ix] = r[ix] + beta * p[ix];
            }
        __syncthreads();
        it++;
    }
    const double usc = 1.0 / sc;  // exact: sc is a power of two
    for (int row = row0; row < N; row += RS)
        if (cv) z[(size_t)row * C + c] *= usc;
    if (threadIdx.x == 0) {
        atomicMax(it_max, it);
        if (it >= maxit) atomicAdd(noconv, 1);
    }
}

// ----------------------------------------------------------------- dense GEMM
// Y[n][C] = A[n][n] X[n][C] (n = npad, multiple of 32), FP64.
constexpr int GB_M = 64, GB_K = 32, GB_N = 32;
__global__ void __launch_bounds__(256) k_gemm(int n, int K, int C, const double* __restrict__ A,
                                              const double* __restrict__ X, double* __restrict__ Y) {
    // rows n, contraction K (multiple of GB_K), A row-major with lda = K
    __shared__ double sa[GB_M][GB_K + 1];
    __shared__ double sx[GB_K][GB_N];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    const int row0 = blockIdx.x * GB_M, col0 = blockIdx.y * GB_N;
    double acc[8];
#pragma unroll
    for (int i = 0; i < 8; i++) acc[i] = 0.0;
    for (int k0 = 0; k0 < K; k0 += GB_K) {
        for (int e = threadIdx.x; e < GB_M * GB_K; e += 256) {
            const int r = e / GB_K, k = e - r * GB_K;
            sa[r][k] = (row0 + r < n) ? A[(size_t)(row0 + r) * K + k0 + k] : 0.0;
        }
        for (int e = threadIdx.x; e < GB_K * GB_N; e += 256) {
            const int k = e / GB_N, cc = e - k * GB_N;
            sx[k][cc] = (col0 + cc < C) ? X[(size_t)(k0 + k) * C + col0 + cc] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < GB_K; k++) {
            const double xv = sx[k][tx];
#pragma unroll
            for (int i = 0; i < 8; i++) acc[i] = fma(sa[ty + 8 * i][k], xv, acc[i]);
        }
        __syncthreads();
    }
    if (col0 + tx < C) {
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int r = row0 + ty + 8 * i;
            if (r < n) Y[(size_t)r * C + col0 + tx] = acc[i];
        }
    }
}

// Y[n][C] = A[n][n] X[n][C] for C <= 8: one warp per row, lanes over the
// contraction index (coalesced rows of A), warp-shuffle reduction.
template <int CC>
__global__ void __launch_bounds__(256) k_gemv_small(int n, int K, const double* __restrict__ A,
                                                    const double* __restrict__ X, double* __restrict__ Y) {
    const int lane = threadIdx.x & 31;
    for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < n; row += (gridDim.x * blockDim.x) >> 5) {
        double acc[CC];
#pragma unroll
        for (int c = 0; c < CC; c++) acc[c] = 0.0;
        const double* a = A + (size_t)row * K;
        for (int k = lane; k < K; k += 32) {
            const double av = a[k];
#pragma unroll
            for (int c = 0; c < CC; c++) acc[c] = fma(av, X[(size_t)k * CC + c], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < CC; c++) {
            double v = acc[c];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0) Y[(size_t)row * CC + c] = v;
        }
    }
}

// ----------------------------------------------------------------- RHS
// rho1[e][b] (u-part) / rho1[e][B+b] (v-part): (1/dt) int p_i (e, h) tested;
// rho2: (1/T_max) (d/dt^-1 (e, h))(i dt) tested, 0 after t_trunc.
// Testing with n x f_m gives -<f_m, .>. Section V-C, Eq. (hin).
__global__ void k_rhs(int ne, int npad, int B, int nq, const double* __restrict__ xq, const double* __restrict__ wf,
                      const double* __restrict__ waves, double ti, double tprev, double dt, double tmax, double c,
                      double eta, double* __restrict__ rho1, double* __restrict__ rho2) {
    const int C2 = 2 * B;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npad * B; i += gridDim.x * blockDim.x) {
        const int r = i / B, b = i - r * B;
        if (r >= ne) {
            rho1[(size_t)r * C2 + b] = rho1[(size_t)r * C2 + B + b] = 0.0;
            rho2[(size_t)r * C2 + b] = rho2[(size_t)r * C2 + B + b] = 0.0;
            continue;
        }
        const double* wv = waves + 10 * b;
        const double A = wv[0], px = wv[1], py = wv[2], pz = wv[3], kx = wv[4], ky = wv[5], kz = wv[6];
        const double w = wv[7], t0 = wv[8], ttr = wv[9];
        const double hx = (ky * pz - kz * py) / eta, hy = (kz * px - kx * pz) / eta, hz = (kx * py - ky * px) / eta;
        double e1 = 0, h1 = 0, e2 = 0, h2 = 0;
        for (int q = 0; q < nq; q++) {
            const double* x = xq + ((size_t)r * nq + q) * 3;
            const double* f = wf + ((size_t)r * nq + q) * 3;
            const double kd = kx * x[0] + ky * x[1] + kz * x[2];
            const double a1 = (4.0 / w) * (c * (ti - t0) - kd);
            const double a0 = (4.0 / w) * (c * (tprev - t0) - kd);
            const double s1 = (A / (2.0 * c)) * (1.0 + erf(a1));
            const double ds = (A / (2.0 * c)) * (erf(a1) - erf(a0));
            const double fp = f[0] * px + f[1] * py + f[2] * pz;
            const double fh = f[0] * hx + f[1] * hy + f[2] * hz;
            e1 += fp * ds;
            h1 += fh * ds;
            e2 += fp * s1;
            h2 += fh * s1;
        }
        rho1[(size_t)r * C2 + b] = -e1 / dt;
        rho1[(size_t)r * C2 + B + b] = -h1 / dt;
        const bool on = ti <= ttr;
        rho2[(size_t)r * C2 + b] = on ? -e2 / tmax : 0.0;
        rho2[(size_t)r * C2 + B + b] = on ? -h2 / tmax : 0.0;
    }
}

// W_a = sum_{k=a}^{kmax-1} variant-2 loop panel of step i-k (steps >= 1), a = 1..amax
__global__ void k_window(int n, int kmax, int amax, long long step_i, int R, size_t pstride,
                         const double* __restrict__ ring, double* __restrict__ win) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int k = kmax - 1; k >= 1; k--) {
            const long long src = step_i - k;
            if (src >= 1) {
                const int slot = (int)(src % R);
                acc += ring[(((size_t)slot * 2 + 0) * 3 + 2) * pstride + i];
            }
            if (k <= amax) win[(size_t)k * pstride + i] = acc;
        }
    }
}

// Current recovery (Eq. (dis_jm)) and running Fourier sums of the four parts.
__global__ void k_recover(int ne, int npad, int B, long long step_i, int R, double scale,
                          const double* __restrict__ ring, double* __restrict__ cur, int nfreq,
                          const double* __restrict__ omega, double dt, double* __restrict__ dft) {
    const int C2 = 2 * B;
    const size_t ps = (size_t)npad * C2;
    const int slot = (int)(step_i % R), slotp = (int)((step_i - 1) % R);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npad * B; i += gridDim.x * blockDim.x) {
        const int r = i / B, b = i - r * B;
        const double* L = ring + ((size_t)slot * 2 + 0) * 3 * ps;
        const double* S = ring + ((size_t)slot * 2 + 1) * 3 * ps;
        const double* Sp = ring + ((size_t)slotp * 2 + 1) * 3 * ps;
        const double lu = L[(size_t)r * C2 + b], lv = L[(size_t)r * C2 + B + b];
        const double su = S[(size_t)r * C2 + b], sv = S[(size_t)r * C2 + B + b];
        const double spu = step_i >= 2 ? Sp[(size_t)r * C2 + b] : 0.0;
        const double spv = step_i >= 2 ? Sp[(size_t)r * C2 + B + b] : 0.0;
        double q[4] = {lu, scale * (su - spu), lv, scale * (sv - spv)};
        const size_t nb = (size_t)npad * B;
        for (int j = 0; j < 4; j++) cur[j * nb + i] = q[j];
        for (int f = 0; f < nfreq; f++) {
            const double w = omega[f];
            double wr, wi;
            if (w == 0.0) {
                wr = dt;
                wi = 0.0;
            } else {
                // e^{-j w i dt} (e^{j w dt} - 1) / (j w)
                double s0, c0, s1, c1;
                sincos(-w * (double)step_i * dt, &s0, &c0);
                sincos(w * dt, &s1, &c1);
                const double ar = c1 - 1.0, ai = s1;          // e^{j w dt} - 1
                const double br = ai / w, bi = -ar / w;       // divided by j w
                wr = c0 * br - s0 * bi;
                wi = c0 * bi + s0 * br;
            }
            double* d = dft + (size_t)f * 4 * nb * 2;
            for (int j = 0; j < 4; j++) {
                d[(j * nb + i) * 2] += q[j] * wr;
                d[(j * nb + i) * 2 + 1] += q[j] * wi;
            }
        }
    }
}

// out[b][part][m] = x[iperm[m]][part*B + b]
__global__ void k_pack_w(int ne, int B, const int* __restrict__ iperm, const double* __restrict__ x,
                         double* __restrict__ out) {
    const int C2 = 2 * B;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B * 2 * ne; i += gridDim.x * blockDim.x) {
        const int b = i / (2 * ne), rem = i - b * 2 * ne, part = rem / ne, m = rem - part * ne;
        out[i] = x[(size_t)iperm[m] * C2 + part * B + b];
    }
}

// ----------------------------------------------------------------- GMRES
// System b of the batch uses columns b and B+b of a block vector.
// partial[chunk][v][b] = sum over the chunk's rows of <V_v, w>_b
constexpr int GM_ROWS = 256;
__global__ void k_gm_dots(int npad, int B, const double* __restrict__ V, size_t vstride, int nvec,
                          const double* __restrict__ w, double* __restrict__ partial) {
    const int C2 = 2 * B;
    const int v = blockIdx.y;
    const int r0 = blockIdx.x * GM_ROWS;
    const double* Vv = V + (size_t)v * vstride;
    __shared__ double sred[256];
    // thread layout: column b = tid % B, row sub = tid / B
    const int b = threadIdx.x % B, rs = threadIdx.x / B, RS = blockDim.x / B;
    double s = 0.0;
    if (threadIdx.x < RS * B)
        for (int r = r0 + rs; r < min(r0 + GM_ROWS, npad); r += RS) {
            const size_t ix = (size_t)r * C2 + b;
            s = fma(Vv[ix], w[ix], s);
            s = fma(Vv[ix + B], w[ix + B], s);
        }
    sred[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < B) {
        double t = 0.0;
        for (int k = 0; k < RS; k++) t += sred[k * B + threadIdx.x];
        partial[((size_t)blockIdx.x * nvec + v) * B + threadIdx.x] = t;
    }
}

__global__ void k_gm_dots_reduce(int nchunk, int nvec, int B, const double* __restrict__ partial,
                                 double* __restrict__ out, int do_sqrt) {
    for (int i = threadIdx.x; i < nvec * B; i += blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < nchunk; c++) s += partial[(size_t)c * nvec * B + i];
        out[i] = do_sqrt ? sqrt(s) : s;
    }
}

// w[r][c] -= sum_v V_v[r][c] coef[v][b(c)]  (sign = -1) or x += V y (sign = +1)
__global__ void k_gm_update(int npad, int B, const double* __restrict__ V, size_t vstride, int nvec,
                            const double* __restrict__ coef, double sign, double* __restrict__ w) {
    const int C2 = 2 * B;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npad * C2; i += gridDim.x * blockDim.x) {
        const int c = i % C2, b = c % B;
        double s = 0.0;
        for (int v = 0; v < nvec; v++) s = fma(V[(size_t)v * vstride + i], coef[v * B + b], s);
        w[i] += sign * s;
    }
}

__global__ void k_gm_scale(int npad, int B, const double* __restrict__ w, const double* __restrict__ nrm,
                           const int* __restrict__ active, double* __restrict__ v) {
    const int C2 = 2 * B;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npad * C2; i += gridDim.x * blockDim.x) {
        const int b = (i % C2) % B;
        const double d = nrm[b];
        v[i] = (active[b] && d > 0.0) ? w[i] / d : 0.0;
    }
}

// Per wave b (the u and v columns b and B + b of a block vector): sc[b] =
// 2^-e, 2^e the power of two at or below max |x| over both columns (1 when
// x is zero). One CTA per wave.
__global__ void k_wave_scale(int npad, int B, const double* __restrict__ x, double* __restrict__ sc) {
    __shared__ double red[256];
    const int b = blockIdx.x, C2 = 2 * B;
    double m = 0.0;
    for (int i = threadIdx.x; i < 2 * npad; i += blockDim.x) {
        const int row = i >> 1, col = (i & 1) ? B + b : b;
        m = fmax(m, fabs(x[(size_t)row * C2 + col]));
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) sc[b] = red[0] > 0.0 ? ldexp(1.0, -ilogb(red[0])) : 1.0;
}

// x[:, b] and x[:, B + b] times sc[b] (inverse: divided by it; exact, powers of two)
__global__ void k_wave_apply(int npad, int B, const double* __restrict__ sc, int inverse, double* __restrict__ x) {
    const int C2 = 2 * B;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npad * C2; i += gridDim.x * blockDim.x) {
        const double f = sc[(i % C2) % B];
        x[i] = inverse ? x[i] / f : x[i] * f;
    }
}

// gstate layout per system b: H[(m+1) x m], g[m+1], cs[m], sn[m]
__global__ void k_gm_init(int B, int m, const double* __restrict__ beta, double* __restrict__ H,
                          double* __restrict__ g, int* __restrict__ active, int* __restrict__ jend,
                          double* __restrict__ bnorm, int first_cycle, double* __restrict__ resid) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    for (int i = 0; i <= m; i++) g[(size_t)b * (m + 1) + i] = 0.0;
    g[(size_t)b * (m + 1)] = beta[b];
    if (first_cycle) bnorm[b] = beta[b];
    const double bn = bnorm[b];
    active[b] = (beta[b] > 0.0 && bn > 0.0) ? 1 : 0;
    jend[b] = 0;
    if (resid) resid[b] = bn > 0.0 ? beta[b] / bn : 0.0;
}

__global__ void k_gm_arnoldi(int B, int m, int j, const double* __restrict__ hcol, const double* __restrict__ nrm,
                             double* __restrict__ H, double* __restrict__ g, double* __restrict__ cs,
                             double* __restrict__ sn, int* __restrict__ active, int* __restrict__ jend,
                             const double* __restrict__ bnorm, double tol, double* __restrict__ resid) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    double* Hb = H + (size_t)b * (m + 1) * m;
    double* gb = g + (size_t)b * (m + 1);
    double* cb = cs + (size_t)b * m;
    double* sb = sn + (size_t)b * m;
    if (!active[b]) return;
    for (int i = 0; i <= j; i++) Hb[i * m + j] = hcol[i * B + b];
    Hb[(j + 1) * m + j] = nrm[b];
    for (int i = 0; i < j; i++) {
        const double a = Hb[i * m + j], c2 = Hb[(i + 1) * m + j];
        Hb[i * m + j] = cb[i] * a + sb[i] * c2;
        Hb[(i + 1) * m + j] = -sb[i] * a + cb[i] * c2;
    }
    const double a = Hb[j * m + j], c2 = Hb[(j + 1) * m + j];
    const double d = hypot(a, c2);
    double cc = 1.0, ss = 0.0;
    if (d > 0.0) {
        cc = a / d;
        ss = c2 / d;
    }
    cb[j] = cc;
    sb[j] = ss;
    Hb[j * m + j] = d;
    Hb[(j + 1) * m + j] = 0.0;
    gb[j + 1] = -ss * gb[j];
    gb[j] = cc * gb[j];
    const double rr = fabs(gb[j + 1]) / bnorm[b];
    resid[b] = rr;
    jend[b] = j + 1;
    if (rr <= tol || !(nrm[b] > 0.0)) active[b] = 0;
}

// y = H^{-1} g (upper triangular, size jend[b]) into y[i][b]
__global__ void k_gm_backsolve(int B, int m, const double* __restrict__ H, const double* __restrict__ g,
                               const int* __restrict__ jend, double* __restrict__ y) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const double* Hb = H + (size_t)b * (m + 1) * m;
    const double* gb = g + (size_t)b * (m + 1);
    const int n = jend[b];
    for (int i = 0; i < m; i++) y[i * B + b] = 0.0;
    for (int i = n - 1; i >= 0; i--) {
        double s = gb[i];
        for (int k = i + 1; k < n; k++) s -= Hb[i * m + k] * y[k * B + b];
        y[i * B + b] = Hb[i * m + i] != 0.0 ? s / Hb[i * m + i] : 0.0;
    }
}


// out[r][0..C) = a[r], out[r][C..2C) = b[r]
__global__ void k_pack2(int n, int C, const double* __restrict__ a, const double* __restrict__ b,
                        double* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * 2 * C; i += gridDim.x * blockDim.x) {
        const int r = i / (2 * C), c = i - r * 2 * C;
        out[i] = c < C ? a[(size_t)r * C + c] : b[(size_t)r * C + c - C];
    }
}

// q1 = X[:, :C] - P[:, :C] (= P^{SH} x1),  q2 = P[:, C:] (= P^L x2)
__global__ void k_unpack_q(int n, int C, const double* __restrict__ X, const double* __restrict__ P,
                           double* __restrict__ q1, double* __restrict__ q2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * C; i += gridDim.x * blockDim.x) {
        const int r = i / C, c = i - r * C;
        q1[i] = X[(size_t)r * 2 * C + c] - P[(size_t)r * 2 * C + c];
        q2[i] = P[(size_t)r * 2 * C + C + c];
    }
}

// out[b][j][m] = cur[j][iperm[m]][b]
__global__ void k_pack_cur(int ne, int npad, int B, const int* __restrict__ iperm, const double* __restrict__ cur,
                           double* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B * 4 * ne; i += gridDim.x * blockDim.x) {
        const int b = i / (4 * ne), rem = i - b * 4 * ne, j = rem / ne, m = rem - j * ne;
        out[i] = cur[((size_t)j * npad + iperm[m]) * B + b];
    }
}

// Far field E_inf(r) = (j k / 4 pi) [eta r x (r x N) + r x L] / S(w) for every
// (direction, frequency, wave); N, L from the Fourier sums of j and m (loop and
// star parts summed here, after separate accumulation). One CTA per output.
__global__ void k_far_field(int ne, int npad, int B, int nq, int nfreq, int ndir, const double* __restrict__ xq,
                            const double* __restrict__ wf, const double* __restrict__ dft,
                            const double* __restrict__ omega, const double* __restrict__ dirs,
                            const double* __restrict__ waves, double c, double eta, double* __restrict__ E) {
    const int o = blockIdx.x;
    const int d = o % ndir, f = (o / ndir) % nfreq, b = o / (ndir * nfreq);
    const double w = omega[f], k = w / c;
    const double rx = dirs[3 * d], ry = dirs[3 * d + 1], rz = dirs[3 * d + 2];
    const size_t nb = (size_t)npad * B;
    const double* D = dft + (size_t)f * 4 * nb * 2;
    double acc[12];
    for (int j = 0; j < 12; j++) acc[j] = 0.0;
    for (int r = threadIdx.x; r < ne; r += blockDim.x) {
        const size_t ix = (size_t)r * B + b;
        const double jr = D[(0 * nb + ix) * 2] + D[(1 * nb + ix) * 2];
        const double ji = D[(0 * nb + ix) * 2 + 1] + D[(1 * nb + ix) * 2 + 1];
        const double mr = D[(2 * nb + ix) * 2] + D[(3 * nb + ix) * 2];
        const double mi = D[(2 * nb + ix) * 2 + 1] + D[(3 * nb + ix) * 2 + 1];
        for (int q = 0; q < nq; q++) {
            const double* x = xq + ((size_t)r * nq + q) * 3;
            const double* fv = wf + ((size_t)r * nq + q) * 3;
            double sp, cp;
            sincos(k * (rx * x[0] + ry * x[1] + rz * x[2]), &sp, &cp);
            const double ar = jr * cp - ji * sp, ai = jr * sp + ji * cp;
            const double br = mr * cp - mi * sp, bi = mr * sp + mi * cp;
            for (int t = 0; t < 3; t++) {
                acc[2 * t] += ar * fv[t];
                acc[2 * t + 1] += ai * fv[t];
                acc[6 + 2 * t] += br * fv[t];
                acc[6 + 2 * t + 1] += bi * fv[t];
            }
        }
    }
    __shared__ double red[12][256];
    for (int j = 0; j < 12; j++) red[j][threadIdx.x] = acc[j];
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st)
            for (int j = 0; j < 12; j++) red[j][threadIdx.x] += red[j][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double r[3] = {rx, ry, rz};
        double out[6];
        for (int part = 0; part < 2; part++) {  // real, imag
            double N[3], Lv[3];
            for (int t = 0; t < 3; t++) {
                N[t] = red[2 * t + part][0];
                Lv[t] = red[6 + 2 * t + part][0];
            }
            const double rN = r[0] * N[0] + r[1] * N[1] + r[2] * N[2];
            // r x (r x N) = r (r.N) - N ; r x L
            const double rxL[3] = {r[1] * Lv[2] - r[2] * Lv[1], r[2] * Lv[0] - r[0] * Lv[2],
                                   r[0] * Lv[1] - r[1] * Lv[0]};
            for (int t = 0; t < 3; t++) out[2 * t + part] = eta * (r[t] * rN - N[t]) + rxL[t];
        }
        // multiply by j k / (4 pi) and divide by S = (A/c) e^{-j w t0} exp(-(w w_p / 8c)^2)
        const double* wv = waves + 10 * b;
        const double A = wv[0], wp = wv[7], t0 = wv[8];
        const double mag = (A / c) * exp(-(w * wp / (8.0 * c)) * (w * wp / (8.0 * c)));
        double ss, cs;
        sincos(-w * t0, &ss, &cs);
        const double Sr = mag * cs, Si = mag * ss;
        const double den = Sr * Sr + Si * Si;
        const double fac = k / (4.0 * 3.14159265358979323846);
        for (int t = 0; t < 3; t++) {
            const double vr = -fac * out[2 * t + 1], vi = fac * out[2 * t];  // j k/(4 pi) * (vr + j vi)
            const double er = den > 0 ? (vr * Sr + vi * Si) / den : 0.0;
            const double ei = den > 0 ? (vi * Sr - vr * Si) / den : 0.0;
            E[((size_t)o * 3 + t) * 2] = er;
            E[((size_t)o * 3 + t) * 2 + 1] = ei;
        }
    }
}

inline int grid_for(long long n, int bs = 256) {
    long long g = (n + bs - 1) / bs;
    if (g > 65535LL * 8) g = 65535LL * 8;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

namespace mot {

void launch_axpby(mot_handle* h, int n, double a, const double* x, double b, const double* y, double* z,
                  cudaStream_t s) {
    k_axpby<<<grid_for(n), 256, 0, s>>>(n, a, x, b, y, z);
    h->launches++;
}

void launch_variants(mot_handle* h, const double* x, double* dst, double eta, double etap, cudaStream_t s) {
    k_variants<<<grid_for((long long)h->npad * h->B), 256, 0, s>>>(h->npad, h->B, x, dst, eta, etap);
    h->launches++;
}

void launch_sigma_t(mot_handle* h, const double* x, int C, double* f, cudaStream_t s) {
    k_sigma_t<<<grid_for((long long)h->nf * C), 256, 0, s>>>(h->nf, C, h->d_face_edges, h->d_face_sgn, x, f);
    h->launches++;
}

void launch_sigma(mot_handle* h, const double* z, int C, double* x, cudaStream_t s) {
    k_sigma<<<grid_for((long long)h->ne * C), 256, 0, s>>>(h->ne, C, h->d_edge_faces, z, x);
    h->launches++;
}

void launch_lambda_t(mot_handle* h, const double* x, int C, double* v, cudaStream_t s) {
    const DCsr& A = h->vtx_edges;
    k_spmv<<<grid_for((long long)A.n * C), 256, 0, s>>>(A.n, C, A.rowptr, A.col, A.val, x, v);
    h->launches++;
}

void launch_lambda(mot_handle* h, const double* z, int C, double* x, cudaStream_t s) {
    k_lambda<<<grid_for((long long)h->ne * C), 256, 0, s>>>(h->ne, C, h->d_edge_verts, z, x);
    h->launches++;
}

void launch_spmv(mot_handle* h, const DCsr& A, const double* x, int C, double* y, cudaStream_t s) {
    k_spmv<<<grid_for((long long)A.n * C), 256, 0, s>>>(A.n, C, A.rowptr, A.col, A.val, x, y);
    h->launches++;
}

int launch_cg(mot_handle* h, const DCsr& A, const DCsr* A2, const double* f, int C, double* z, double* work,
              cudaStream_t s) {
    const int N = A.n;
    double* r = work;
    double* p = r + (size_t)N * C;
    double* q = p + (size_t)N * C;
    double* t = q + (size_t)N * C;
    int cw = 1;
    while (cw < 32 && (C + cw - 1) / cw > 128) cw *= 2;
    const int grid = (C + cw - 1) / cw;
    CsrV a{A.rowptr, A.col, A.val};
    CsrV a2{nullptr, nullptr, nullptr};
    if (A2) a2 = CsrV{A2->rowptr, A2->col, A2->val};
    const double tol = h->opt.cg_tol;
    const int mi = h->opt.cg_maxit;
    int* itmax = h->d_cg_iters;
    int* nc = h->d_cg_iters + 1;
#define MOT_CG_CASE(W)                                                                                         \
    case W:                                                                                                    \
        if (A2)                                                                                                \
            k_cg<W, true><<<grid, 1024, 0, s>>>(N, C, a, a2, f, z, r, p, q, t, tol, mi, itmax, nc);            \
        else                                                                                                   \
            k_cg<W, false><<<grid, 1024, 0, s>>>(N, C, a, a2, f, z, r, p, q, t, tol, mi, itmax, nc);           \
        break;
    switch (cw) {
        MOT_CG_CASE(1)
        MOT_CG_CASE(2)
        MOT_CG_CASE(4)
        MOT_CG_CASE(8)
        MOT_CG_CASE(16)
        MOT_CG_CASE(32)
    }
#undef MOT_CG_CASE
    h->launches++;
    return 0;
}

void launch_gemm_rect(mot_handle* h, int M, int K, const double* A, const double* X, int C, double* Y,
                      cudaStream_t s) {
    if (C <= 8) {
        const int g = grid_for((long long)M * 32);
        switch (C) {
            case 1: k_gemv_small<1><<<g, 256, 0, s>>>(M, K, A, X, Y); break;
            case 2: k_gemv_small<2><<<g, 256, 0, s>>>(M, K, A, X, Y); break;
            case 4: k_gemv_small<4><<<g, 256, 0, s>>>(M, K, A, X, Y); break;
            case 6: k_gemv_small<6><<<g, 256, 0, s>>>(M, K, A, X, Y); break;
            case 8: k_gemv_small<8><<<g, 256, 0, s>>>(M, K, A, X, Y); break;
            default: goto general;
        }
        h->launches++;
        return;
    }
general:
    dim3 grid((M + GB_M - 1) / GB_M, (C + GB_N - 1) / GB_N);
    k_gemm<<<grid, 256, 0, s>>>(M, K, C, A, X, Y);
    h->launches++;
}

void launch_gemm(mot_handle* h, const double* A, const double* X, int C, double* Y, cudaStream_t s) {
    launch_gemm_rect(h, h->npad, h->npad, A, X, C, Y, s);
}

void launch_rhs(mot_handle* h, long long i, double* rho1, double* rho2, cudaStream_t s) {
    k_rhs<<<grid_for((long long)h->npad * h->B), 256, 0, s>>>(h->ne, h->npad, h->B, h->nq, h->d_rhs_x, h->d_rhs_wf,
                                                              h->d_waves, i * h->dt, (i - 1) * h->dt, h->dt,
                                                              h->tmax, h->c, h->eta, rho1, rho2);
    h->launches++;
}

void launch_window_sums(mot_handle* h, long long i, cudaStream_t s) {
    if (h->max_tail_lag < 1) return;
    const size_t ps = (size_t)h->npad * 2 * h->B;
    k_window<<<grid_for((long long)ps), 256, 0, s>>>((int)ps, h->kmax, h->max_tail_lag, i, h->R, ps, h->d_ring,
                                                     h->d_win);
    h->launches++;
}

void launch_recover(mot_handle* h, long long i, cudaStream_t s) {
    k_recover<<<grid_for((long long)h->npad * h->B), 256, 0, s>>>(h->ne, h->npad, h->B, i, h->R, h->tmax / h->dt,
                                                                  h->d_ring, h->d_cur, h->nfreq, h->d_omega, h->dt,
                                                                  h->d_dft);
    h->launches++;
}

void launch_pack_w(mot_handle* h, const double* x, double* out, cudaStream_t s) {
    k_pack_w<<<grid_for((long long)h->B * 2 * h->ne), 256, 0, s>>>(h->ne, h->B, h->d_iperm, x, out);
    h->launches++;
}

void launch_gm_dots(mot_handle* h, const double* V, int nvec, const double* w, double* out, cudaStream_t s) {
    const int nchunk = (h->npad + GM_ROWS - 1) / GM_ROWS;
    dim3 grid(nchunk, nvec);
    k_gm_dots<<<grid, 256, 0, s>>>(h->npad, h->B, V, (size_t)h->npad * 2 * h->B, nvec, w, h->d_red);
    k_gm_dots_reduce<<<1, 256, 0, s>>>(nchunk, nvec, h->B, h->d_red, out, 0);
    h->launches += 2;
}

void launch_gm_norm(mot_handle* h, const double* w, double* out, cudaStream_t s) {
    const int nchunk = (h->npad + GM_ROWS - 1) / GM_ROWS;
    dim3 grid(nchunk, 1);
    k_gm_dots<<<grid, 256, 0, s>>>(h->npad, h->B, w, 0, 1, w, h->d_red);
    k_gm_dots_reduce<<<1, 256, 0, s>>>(nchunk, 1, h->B, h->d_red, out, 1);
    h->launches += 2;
}

void launch_gm_update(mot_handle* h, const double* V, int nvec, const double* coef, double* w, cudaStream_t s) {
    const long long n = (long long)h->npad * 2 * h->B;
    k_gm_update<<<grid_for(n), 256, 0, s>>>(h->npad, h->B, V, (size_t)n, nvec, coef, -1.0, w);
    h->launches++;
}

void launch_gm_scale(mot_handle* h, const double* w, const double* nrm, double* v, cudaStream_t s) {
    const long long n = (long long)h->npad * 2 * h->B;
    k_gm_scale<<<grid_for(n), 256, 0, s>>>(h->npad, h->B, w, nrm, h->d_gm_active, v);
    h->launches++;
}

void launch_wave_scale(mot_handle* h, const double* x, double* sc, cudaStream_t s) {
    k_wave_scale<<<h->B, 256, 0, s>>>(h->npad, h->B, x, sc);
    h->launches++;
}

void launch_wave_apply(mot_handle* h, const double* sc, bool inverse, double* x, cudaStream_t s) {
    const long long n = (long long)h->npad * 2 * h->B;
    k_wave_apply<<<grid_for(n), 256, 0, s>>>(h->npad, h->B, sc, inverse ? 1 : 0, x);
    h->launches++;
}

void launch_gm_init(mot_handle* h, const double* beta, int first_cycle, cudaStream_t s) {
    k_gm_init<<<1, 64, 0, s>>>(h->B, h->gm_m, beta, h->d_H, h->d_g, h->d_gm_active, h->d_gm_jend, h->d_gm_bnorm,
                               first_cycle, h->d_resid);
    h->launches++;
}

void launch_gm_arnoldi_finish(mot_handle* h, int j, const double* hcol, const double* nrm, cudaStream_t s) {
    k_gm_arnoldi<<<1, 64, 0, s>>>(h->B, h->gm_m, j, hcol, nrm, h->d_H, h->d_g, h->d_cs, h->d_sn, h->d_gm_active,
                                  h->d_gm_jend, h->d_gm_bnorm, h->gm_tol, h->d_resid);
    h->launches++;
}

void launch_gm_solve_update(mot_handle* h, double* y, double* x, cudaStream_t s) {
    k_gm_backsolve<<<1, 64, 0, s>>>(h->B, h->gm_m, h->d_H, h->d_g, h->d_gm_jend, y);
    const long long n = (long long)h->npad * 2 * h->B;
    k_gm_update<<<grid_for(n), 256, 0, s>>>(h->npad, h->B, h->d_V, (size_t)n, h->gm_m, y, 1.0, x);
    h->launches += 2;
}


void launch_pack2(mot_handle* h, const double* a, const double* b, int C, double* out, cudaStream_t s) {
    k_pack2<<<grid_for((long long)h->npad * 2 * C), 256, 0, s>>>(h->npad, C, a, b, out);
    h->launches++;
}

void launch_unpack_q(mot_handle* h, const double* X, const double* P, int C, double* q1, double* q2, cudaStream_t s) {
    k_unpack_q<<<grid_for((long long)h->npad * C), 256, 0, s>>>(h->npad, C, X, P, q1, q2);
    h->launches++;
}

void launch_pack_cur(mot_handle* h, double* out, cudaStream_t s) {
    k_pack_cur<<<grid_for((long long)h->B * 4 * h->ne), 256, 0, s>>>(h->ne, h->npad, h->B, h->d_iperm, h->d_cur, out);
    h->launches++;
}

void launch_far_field(mot_handle* h, int n_dir, const double* dirs, double* E, cudaStream_t s) {
    const int n = h->B * h->nfreq * n_dir;
    if (n == 0) return;
    k_far_field<<<n, 256, 0, s>>>(h->ne, h->npad, h->B, h->nq, h->nfreq, n_dir, h->d_rhs_x, h->d_rhs_wf, h->d_dft,
                                  h->d_omega, dirs, h->d_waves, h->c, h->eta, E);
    h->launches++;
}

}  // namespace mot
