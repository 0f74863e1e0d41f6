// Kernels of the mixed-precision MOT path: FP32 history tiles and coefficient
// panels with FP32 products summed in FP64 across tiles, a dense FP32 x FP32
// -> FP64 GEMM for the precomputed Q_0 and left factors, and the load-time
// helpers that assemble those dense matrices column by column from the FP64
// product form.
#include <algorithm>

#include "mot_internal.h"

namespace {

constexpr int T = MOT_TILE;
constexpr int NT = 256;
constexpr int MAXO = T * 2 * MOT_MAX_B / NT;  // 16 outputs per thread per target
constexpr int FLUSH = 4;                     // tiles summed in FP32 before an FP64 flush

__device__ __forceinline__ const float* panel_ptr32(int mode, const float* ring, const float* win, const float* kry,
                                                    long long step_i, int R, int npad, int C2, int k, int part,
                                                    int variant) {
    const size_t ps = (size_t)npad * C2;
    if (mode == 1) return kry + ((size_t)part * 3 + variant) * ps;
    if (part == 2) return win + (size_t)k * ps;
    const int slot = (int)((step_i - k) % R);
    return ring + (((size_t)slot * 2 + part) * 3 + variant) * ps;
}

__global__ void __launch_bounds__(NT) k_hist_f32(const HistTask* __restrict__ tasks,
                                                 const HistChunk* __restrict__ chunks,
                                                 const float* __restrict__ tiles, const float* __restrict__ ring,
                                                 const float* __restrict__ win, const float* __restrict__ kry,
                                                 int mode, long long step_i, int R, int npad, int C2,
                                                 const int* __restrict__ colidx, double* __restrict__ partial) {
    __shared__ float st[T * (T + 1)];
    __shared__ float sp[T * 2 * MOT_MAX_B];
    const HistChunk ch = chunks[blockIdx.x];
    const int nout = T * C2;
    const int tid = threadIdx.x;
    float a0[MAXO], a1[MAXO];
    double d0[MAXO], d1[MAXO];
#pragma unroll
    for (int j = 0; j < MAXO; j++) {
        a0[j] = a1[j] = 0.f;
        d0[j] = d1[j] = 0.0;
    }
    int pending = 0;
    for (int t = ch.first; t < ch.first + ch.count; t++) {
        const HistTask tk = tasks[t];
        const int part = tk.code & 3, variant = (tk.code >> 2) & 3, out = (tk.code >> 4) & 1;
        if (mode == 0 && step_i - tk.k < 1) continue;
        const float* pan = panel_ptr32(mode, ring, win, kry, step_i, R, npad, C2, tk.k, part, variant);
        const int* cols = colidx + (size_t)ch.rb * npad + (size_t)tk.cb * T;
        const float* tl = tiles + (size_t)tk.tile * T * T;
        __syncthreads();
        for (int e = tid; e < T * T; e += NT) st[(e / T) * (T + 1) + (e % T)] = tl[e];
        for (int e = tid; e < T * C2; e += NT) {
            const int r = e / C2;
            sp[e] = pan[(size_t)cols[r] * C2 + (e - r * C2)];
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < MAXO; j++) {
            const int o = tid + j * NT;
            if (o < nout) {
                const int r = o / C2, c = o - r * C2;
                float s = 0.f;
#pragma unroll 8
                for (int n = 0; n < T; n++) s = fmaf(st[r * (T + 1) + n], sp[n * C2 + c], s);
                if (out == 0)
                    a0[j] += s;
                else
                    a1[j] += s;
            }
        }
        if (++pending == FLUSH) {
            pending = 0;
#pragma unroll
            for (int j = 0; j < MAXO; j++) {
                d0[j] += (double)a0[j];
                d1[j] += (double)a1[j];
                a0[j] = a1[j] = 0.f;
            }
        }
    }
    double* dst = partial + (size_t)blockIdx.x * 2 * nout;
#pragma unroll
    for (int j = 0; j < MAXO; j++) {
        const int o = tid + j * NT;
        if (o < nout) {
            dst[o] = d0[j] + (double)a0[j];
            dst[nout + o] = d1[j] + (double)a1[j];
        }
    }
}

// Batched variant for 2B = 128 columns: 128 threads, each owning a 4 x 8 block
// of the 32 x 128 output; tile and gathered panel rows double-buffered with
// cp.async; FP32 register sums added into FP64 shared-memory accumulators when
// the output target changes or every FLUSH tiles.
constexpr int V2_C = 128, V2_AS = T + 4, V2_BS = V2_C + 4;

__device__ __forceinline__ void cp16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }

__global__ void __launch_bounds__(128) k_hist_f32_b128(const HistTask* __restrict__ tasks,
                                                      const HistChunk* __restrict__ chunks,
                                                      const float* __restrict__ tiles, const float* __restrict__ ring,
                                                      const float* __restrict__ win, long long step_i, int R,
                                                      int npad, const int* __restrict__ colidx,
                                                      double* __restrict__ partial) {
    extern __shared__ __align__(16) unsigned char smraw[];
    double* acc64 = reinterpret_cast<double*>(smraw);                    // [2][T][V2_C]
    float* sA = reinterpret_cast<float*>(smraw + sizeof(double) * 2 * T * V2_C);  // [2][T][V2_AS]
    float* sB = sA + 2 * T * V2_AS;                                      // [2][T][V2_BS]
    const HistChunk ch = chunks[blockIdx.x];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;  // columns tx*8..+7, rows ty*4..+3
    for (int e = tid; e < 2 * T * V2_C; e += 128) acc64[e] = 0.0;
    // compact the live tasks of this chunk: skip history before step 1
    auto live = [&](int t) { return step_i - tasks[t].k >= 1; };
    auto issue = [&](int t, int buf) {
        const HistTask tk = tasks[t];
        const int part = tk.code & 3, variant = (tk.code >> 2) & 3;
        const float* pan = panel_ptr32(0, ring, win, nullptr, step_i, R, npad, V2_C, tk.k, part, variant);
        const int* cols = colidx + (size_t)ch.rb * npad + (size_t)tk.cb * T;
        const float* tl = tiles + (size_t)tk.tile * T * T;
        float* a = sA + buf * T * V2_AS;
        float* b = sB + buf * T * V2_BS;
        for (int e = tid; e < T * (T / 4); e += 128) {  // 32 rows x 8 chunks of 16 B
            const int r = e >> 3, c4 = (e & 7) * 4;
            cp16(a + r * V2_AS + c4, tl + r * T + c4);
        }
        for (int e = tid; e < T * (V2_C / 4); e += 128) {  // 32 gathered rows x 32 chunks
            const int r = e >> 5, c4 = (e & 31) * 4;
            cp16(b + r * V2_BS + c4, pan + (size_t)cols[r] * V2_C + c4);
        }
    };
    float acc[4][8];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) acc[i][j] = 0.f;
    int cur_out = -1, pending = 0;
    auto flush = [&]() {
        if (cur_out < 0) return;
        double* d = acc64 + cur_out * T * V2_C;
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 8; j++) {
                d[(ty * 4 + i) * V2_C + tx * 8 + j] += (double)acc[i][j];
                acc[i][j] = 0.f;
            }
        pending = 0;
    };
    const int t_end = ch.first + ch.count;
    int t = ch.first;
    while (t < t_end && !live(t)) t++;
    int buf = 0;
    if (t < t_end) issue(t, 0);
    cp_commit();
    while (t < t_end) {
        int tn = t + 1;
        while (tn < t_end && !live(tn)) tn++;
        if (tn < t_end) issue(tn, buf ^ 1);
        cp_commit();
        cp_wait1();
        __syncthreads();
        const int out = (tasks[t].code >> 4) & 1;
        if (out != cur_out || pending == FLUSH) {
            flush();
            cur_out = out;
        }
        const float* a = sA + buf * T * V2_AS;
        const float* b = sB + buf * T * V2_BS;
#pragma unroll 4
        for (int k = 0; k < T; k++) {
            float av[4];
#pragma unroll
            for (int i = 0; i < 4; i++) av[i] = a[(ty * 4 + i) * V2_AS + k];
            const float4 b0 = *reinterpret_cast<const float4*>(b + k * V2_BS + tx * 8);
            const float4 b1 = *reinterpret_cast<const float4*>(b + k * V2_BS + tx * 8 + 4);
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 8; j++) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        pending++;
        __syncthreads();
        buf ^= 1;
        t = tn;
    }
    cp_wait0();
    flush();
    __syncthreads();
    double* dst = partial + (size_t)blockIdx.x * 2 * T * V2_C;
    for (int e = tid; e < 2 * T * V2_C; e += 128) dst[e] = acc64[e];
}

__global__ void k_hist_reduce2(const int* __restrict__ chunk_ptr, const double* __restrict__ partial, int C2,
                               double* __restrict__ s1, double* __restrict__ s2) {
    const int rb = blockIdx.x;
    const int nout = T * C2;
    const int c0 = chunk_ptr[rb], c1 = chunk_ptr[rb + 1];
    for (int o = threadIdx.x; o < nout; o += blockDim.x) {
        double a = 0.0, b = 0.0;
        for (int c = c0; c < c1; c++) {
            a += partial[(size_t)c * 2 * nout + o];
            b += partial[(size_t)c * 2 * nout + nout + o];
        }
        s1[(size_t)rb * nout + o] = a;
        s2[(size_t)rb * nout + o] = b;
    }
}

// Y[M][N] (double) = A[M][K] (float, row-major, lda = K) * X[K][N] (float).
// 128 x 64 output tile per CTA, 8 x 4 outputs per thread; FP32 products summed
// in FP32 over 128 consecutive k, then added into FP64 accumulators. K is split
// over gridDim.z CTAs (each a multiple of 128 long), so that small-N products
// fill the GPU; with more than one split each CTA writes its FP64 partial
// result to W[z][M][N] and k_sgemm_reduce sums the splits in a fixed order.
constexpr int SG_M = 128, SG_N = 64, SG_K = 16, SG_FLUSH = 128;
__global__ void __launch_bounds__(256) k_sgemm_d(int M, int N, int K, int kchunk, const float* __restrict__ A,
                                                 const float* __restrict__ X, double* __restrict__ Y) {
    __shared__ float sa[2][SG_K][SG_M + 4];
    __shared__ __align__(16) float sx[2][SG_K][SG_N];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;  // 16 x 16 threads: 4 cols x 8 rows each
    const int row0 = blockIdx.x * SG_M, col0 = blockIdx.y * SG_N;
    const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
    float acc[8][4];
    double dacc[8][4];
#pragma unroll
    for (int i = 0; i < 8; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            acc[i][j] = 0.f;
            dacc[i][j] = 0.0;
        }
    // loader mapping: A tile 128 rows x 16 k = 512 float4 (2 per thread, along k);
    // X tile 16 k x 64 cols = 256 float4 (1 per thread, along the columns)
    const bool avec = (K & 3) == 0, xvec = (N & 3) == 0;
    float4 ra[2], rx;
    auto load = [&](int k0) {
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int e = tid + h * 256, r = e >> 2, kq = (e & 3) * 4;
            const int gr = row0 + r, gk = k0 + kq;
            if (gr < M && avec && gk + 3 < kend) {
                ra[h] = __ldg(reinterpret_cast<const float4*>(A + (size_t)gr * K + gk));
            } else {
                float v[4];
#pragma unroll
                for (int q = 0; q < 4; q++) v[q] = (gr < M && gk + q < kend) ? A[(size_t)gr * K + gk + q] : 0.f;
                ra[h] = make_float4(v[0], v[1], v[2], v[3]);
            }
        }
        {
            const int k = tid >> 4, c4 = (tid & 15) * 4;
            const int gk = k0 + k, gc = col0 + c4;
            if (gk < kend && xvec && gc + 3 < N) {
                rx = __ldg(reinterpret_cast<const float4*>(X + (size_t)gk * N + gc));
            } else {
                float v[4];
#pragma unroll
                for (int q = 0; q < 4; q++) v[q] = (gk < kend && gc + q < N) ? X[(size_t)gk * N + gc + q] : 0.f;
                rx = make_float4(v[0], v[1], v[2], v[3]);
            }
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int e = tid + h * 256, r = e >> 2, kq = (e & 3) * 4;
            sa[buf][kq + 0][r] = ra[h].x;
            sa[buf][kq + 1][r] = ra[h].y;
            sa[buf][kq + 2][r] = ra[h].z;
            sa[buf][kq + 3][r] = ra[h].w;
        }
        *reinterpret_cast<float4*>(&sx[buf][tid >> 4][(tid & 15) * 4]) = rx;
    };
    int buf = 0, since = 0;
    if (kbeg < kend) {
        load(kbeg);
        store(0);
    }
    __syncthreads();
    for (int k0 = kbeg; k0 < kend; k0 += SG_K) {
        const bool more = k0 + SG_K < kend;
        if (more) load(k0 + SG_K);  // next tile in flight while this one is used
#pragma unroll
        for (int k = 0; k < SG_K; k++) {
            const float4 a0 = *reinterpret_cast<const float4*>(&sa[buf][k][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&sa[buf][k][ty * 8 + 4]);
            const float4 xv = *reinterpret_cast<const float4*>(&sx[buf][k][tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float xw[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
            for (int i = 0; i < 8; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fmaf(av[i], xw[j], acc[i][j]);
        }
        since += SG_K;
        if (since >= SG_FLUSH) {
            since = 0;
#pragma unroll
            for (int i = 0; i < 8; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    dacc[i][j] += (double)acc[i][j];
                    acc[i][j] = 0.f;
                }
        }
        if (more) store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
    double* out = Y + (size_t)blockIdx.z * M * N;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int r = row0 + ty * 8 + i;
        if (r >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int c = col0 + tx * 4 + j;
            if (c < N) out[(size_t)r * N + c] = dacc[i][j] + (double)acc[i][j];
        }
    }
}

__global__ void k_sgemm_reduce(size_t n, int S, const double* __restrict__ W, double* __restrict__ Y) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int z = 0; z < S; z++) v += W[(size_t)z * n + i];
        Y[i] = v;
    }
}

__global__ void k_d2f(size_t n, const double* __restrict__ x, float* __restrict__ y) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = (float)x[i];
}

// Unit right-hand sides for the column-by-column assembly of a dense operator:
// batch entry b selects column J = J0 + b of the (2 npad)-dimensional space
// (interleaved index 2 q + c: edge q, component c). X is a block vector [npad][2B].
__global__ void k_unit_cols(int npad, int B, long long J0, long long Jend, double* __restrict__ X) {
    const int C2 = 2 * B;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)npad * C2;
         i += (size_t)gridDim.x * blockDim.x) {
        const int q = (int)(i / C2), cc = (int)(i % C2), c = cc / B, b = cc % B;
        const long long J = J0 + b;
        X[i] = (J < Jend && J == 2LL * q + c) ? 1.0 : 0.0;
    }
}

// Dense[(2p+a) * ldd + J0 + b] = Y[p][a*B + b] for J0 + b < Jend (rows 2 npad)
__global__ void k_scatter_cols(int npad, int B, long long J0, long long Jend, const double* __restrict__ Y,
                               double* __restrict__ D, long long ldd) {
    const int C2 = 2 * B;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)npad * C2;
         i += (size_t)gridDim.x * blockDim.x) {
        const int p = (int)(i / C2), cc = (int)(i % C2), a = cc / B, b = cc % B;
        const long long J = J0 + b;
        if (J < Jend) D[(size_t)(2LL * p + a) * ldd + J] = Y[i];
    }
}

// Left-factor columns: batch entry b selects column q = Q0 + b of [M1 | M2]
// (q < npad: unit u-part in y1; npad <= q < 2 npad: unit u-part in y2).
__global__ void k_unit_lf(int npad, int B, long long Q0, long long Qend, double* __restrict__ y1,
                          double* __restrict__ y2) {
    const int C2 = 2 * B;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)npad * C2;
         i += (size_t)gridDim.x * blockDim.x) {
        const int p = (int)(i / C2), cc = (int)(i % C2);
        const long long q = Q0 + (cc % B);
        const bool upart = cc < B;
        y1[i] = (upart && q < Qend && q < npad && q == p) ? 1.0 : 0.0;
        y2[i] = (upart && q < Qend && q >= npad && q - npad == p) ? 1.0 : 0.0;
    }
}

// LF[p * ldd + Q0 + b] = out[p][b] (u-part of the left factor applied to unit columns)
__global__ void k_scatter_lf(int npad, int B, long long Q0, long long Qend, const double* __restrict__ out,
                             double* __restrict__ D, long long ldd) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)npad * B;
         i += (size_t)gridDim.x * blockDim.x) {
        const int p = (int)(i / B), b = (int)(i % B);
        if (Q0 + b < Qend) D[(size_t)p * ldd + Q0 + b] = out[(size_t)p * 2 * B + b];
    }
}

inline int grid_for(size_t n, int bs = 256) {
    size_t g = (n + bs - 1) / bs;
    if (g > 65535ULL * 8) g = 65535ULL * 8;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

namespace mot {

void launch_history32(mot_handle* h, const TaskList& tl, const float* tiles, const float* ring, const float* win,
                      const float* kry, int mode, long long step_i, double* out_s1, double* out_s2,
                      cudaStream_t s) {
    const int C2 = 2 * h->B;
    if (tl.nchunks > 0) {
        const bool timed = h->opt.timing && mode == 0 && h->ev0 && step_i > h->K;
        if (timed) cudaEventRecord(h->ev0, s);
        if (C2 == V2_C && mode == 0) {
            const size_t smem = sizeof(double) * 2 * T * V2_C + sizeof(float) * 2 * T * (V2_AS + V2_BS);
            static std::atomic<unsigned long long> attr{0};
            once_per_device(attr, h->dev, [smem] {
                cudaFuncSetAttribute(k_hist_f32_b128, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            });
            k_hist_f32_b128<<<tl.nchunks, 128, smem, s>>>(tl.tasks, tl.chunks, tiles, ring, win, step_i, h->R,
                                                          h->npad, h->d_colidx, h->d_partial);
        } else {
            k_hist_f32<<<tl.nchunks, NT, 0, s>>>(tl.tasks, tl.chunks, tiles, ring, win, kry, mode, step_i, h->R,
                                                 h->npad, C2, h->d_colidx, h->d_partial);
        }
        if (timed) {
            cudaEventRecord(h->ev1, s);
            h->ev_pending = true;
        }
        h->launches++;
    }
    launch_history_reduce(h, tl, C2, out_s1, out_s2, s);
}

void launch_history_reduce(mot_handle* h, const TaskList& tl, int C2, double* out_s1, double* out_s2,
                           cudaStream_t s) {
    k_hist_reduce2<<<h->nrb, 256, 0, s>>>(tl.chunk_ptr, h->d_partial, C2, out_s1, out_s2);
    h->launches++;
}

void launch_sgemm_d(mot_handle* h, int M, int N, int K, const float* A, const float* X, double* Y, cudaStream_t s) {
    int nsm = 148;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->dev);
    const int tiles = ((M + SG_M - 1) / SG_M) * ((N + SG_N - 1) / SG_N);
    // K splits: about four CTAs per SM, each split a multiple of the FP64 flush length
    int S = std::max(1, std::min((4 * nsm + tiles - 1) / tiles, std::min(16, (K + SG_FLUSH - 1) / SG_FLUSH)));
    const size_t need = (size_t)S * M * N * sizeof(double);
    if (S > 1 && need > h->sgws_bytes) {
        if (h->d_sgws) {
            cudaFree(h->d_sgws);
            h->device_bytes -= (int64_t)h->sgws_bytes;
        }
        h->sgws_bytes = 0;
        h->d_sgws = (double*)dalloc(h, need);
        if (h->d_sgws) h->sgws_bytes = need;
    }
    if (S > 1 && !h->d_sgws) S = 1;  // no workspace: one split
    const int kchunk = ((K + S - 1) / S + SG_FLUSH - 1) / SG_FLUSH * SG_FLUSH;
    S = (K + kchunk - 1) / kchunk;
    dim3 grid((M + SG_M - 1) / SG_M, (N + SG_N - 1) / SG_N, S);
    k_sgemm_d<<<grid, 256, 0, s>>>(M, N, K, kchunk, A, X, S > 1 ? h->d_sgws : Y);
    h->launches++;
    if (S > 1) {
        const size_t n = (size_t)M * N;
        k_sgemm_reduce<<<(int)std::min<size_t>((n + 255) / 256, 4096), 256, 0, s>>>(n, S, h->d_sgws, Y);
        h->launches++;
    }
}

void launch_d2f(mot_handle* h, size_t n, const double* x, float* y, cudaStream_t s) {
    k_d2f<<<grid_for(n), 256, 0, s>>>(n, x, y);
    h->launches++;
}

void launch_unit_cols(mot_handle* h, long long J0, long long Jend, double* X, cudaStream_t s) {
    k_unit_cols<<<grid_for((size_t)h->npad * 2 * h->B), 256, 0, s>>>(h->npad, h->B, J0, Jend, X);
    h->launches++;
}

void launch_scatter_cols(mot_handle* h, long long J0, long long Jend, const double* Y, double* D, long long ldd,
                         cudaStream_t s) {
    k_scatter_cols<<<grid_for((size_t)h->npad * 2 * h->B), 256, 0, s>>>(h->npad, h->B, J0, Jend, Y, D, ldd);
    h->launches++;
}

void launch_unit_lf(mot_handle* h, long long Q0, long long Qend, double* y1, double* y2, cudaStream_t s) {
    k_unit_lf<<<grid_for((size_t)h->npad * 2 * h->B), 256, 0, s>>>(h->npad, h->B, Q0, Qend, y1, y2);
    h->launches++;
}

void launch_scatter_lf(mot_handle* h, long long Q0, long long Qend, const double* out, double* D, long long ldd,
                       cudaStream_t s) {
    k_scatter_lf<<<grid_for((size_t)h->npad * h->B), 256, 0, s>>>(h->npad, h->B, Q0, Qend, out, D, ldd);
    h->launches++;
}

}  // namespace mot
