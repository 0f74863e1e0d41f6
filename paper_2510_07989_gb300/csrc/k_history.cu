// Block-sparse history contraction of the MOT step (paper Eq. (MOT)):
//   s1 = sum_k A_k l_{i-k} + A^_k s_{i-k},   s2 = sum_k A~_k l_{i-k} + A_k s_{i-k}
// where each family is the 2x2 PMCHWT block of Section V-B built from stored
// T, T', K + K' matrices. The medium factors (eta, eta') and the block signs of
// the 2x2 structure are folded into three precomputed variants of every
// coefficient panel, so every stored tile is a plain (TILE x TILE) * (TILE x 2B)
// product accumulated into one of two outputs.
//
// FP64 path: one CTA per chunk of tile tasks of a single row block; partial sums
// go to a scratch buffer and a second kernel reduces the chunks of each row
// block in a fixed order (deterministic).
#include "mot_internal.h"

namespace {

constexpr int T = MOT_TILE;
constexpr int NT = 256;                       // threads per CTA
constexpr int MAXO = T * 2 * MOT_MAX_B / NT;  // outputs per thread per target (16)

__device__ __forceinline__ const double* panel_ptr(int mode, const double* ring, const double* win,
                                                   const double* kry, long long step_i, int R, int npad,
                                                   int C2, int k, int part, int variant) {
    const size_t pstride = (size_t)npad * C2;
    if (mode == 1) return kry + ((size_t)part * 3 + variant) * pstride;
    if (part == 2) return win + (size_t)k * pstride;
    long long src = step_i - k;
    int slot = (int)(src % R);
    return ring + (((size_t)slot * 2 + part) * 3 + variant) * pstride;
}

__global__ void __launch_bounds__(NT) k_hist_f64(const HistTask* __restrict__ tasks,
                                                 const HistChunk* __restrict__ chunks,
                                                 const double* __restrict__ tiles, const double* __restrict__ ring,
                                                 const double* __restrict__ win, const double* __restrict__ kry,
                                                 int mode, long long step_i, int R, int npad, int C2,
                                                 const int* __restrict__ colidx, double* __restrict__ partial) {
    extern __shared__ double sm[];
    double* st = sm;                  // T x (T + 1)
    double* sp = st + T * (T + 1);    // T x C2
    const HistChunk ch = chunks[blockIdx.x];
    const int nout = T * C2;
    const int tid = threadIdx.x;
    double acc0[MAXO], acc1[MAXO];
#pragma unroll
    for (int j = 0; j < MAXO; j++) {
        acc0[j] = 0.0;
        acc1[j] = 0.0;
    }
    for (int t = ch.first; t < ch.first + ch.count; t++) {
        const HistTask tk = tasks[t];
        const int part = tk.code & 3, variant = (tk.code >> 2) & 3, out = (tk.code >> 4) & 1;
        if (mode == 0 && step_i - tk.k < 1) continue;  // history before step 1 is zero
        const double* pan = panel_ptr(mode, ring, win, kry, step_i, R, npad, C2, tk.k, part, variant);
        const int* cols = colidx + (size_t)ch.rb * npad + (size_t)tk.cb * T;  // distance-sorted columns
        const double* tl = tiles + (size_t)tk.tile * T * T;
        __syncthreads();
        for (int e = tid; e < T * T; e += NT) st[(e / T) * (T + 1) + (e % T)] = tl[e];
        for (int e = tid; e < T * C2; e += NT) {
            const int r = e / C2;
            sp[e] = pan[(size_t)cols[r] * C2 + (e - r * C2)];
        }
        __syncthreads();
        if (out == 0) {
#pragma unroll
            for (int j = 0; j < MAXO; j++) {
                const int o = tid + j * NT;
                if (o < nout) {
                    const int r = o / C2, c = o - r * C2;
                    double s = acc0[j];
#pragma unroll 8
                    for (int n = 0; n < T; n++) s = fma(st[r * (T + 1) + n], sp[n * C2 + c], s);
                    acc0[j] = s;
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < MAXO; j++) {
                const int o = tid + j * NT;
                if (o < nout) {
                    const int r = o / C2, c = o - r * C2;
                    double s = acc1[j];
#pragma unroll 8
                    for (int n = 0; n < T; n++) s = fma(st[r * (T + 1) + n], sp[n * C2 + c], s);
                    acc1[j] = s;
                }
            }
        }
    }
    double* dst = partial + (size_t)blockIdx.x * 2 * nout;
#pragma unroll
    for (int j = 0; j < MAXO; j++) {
        const int o = tid + j * NT;
        if (o < nout) {
            dst[o] = acc0[j];
            dst[nout + o] = acc1[j];
        }
    }
}

// out_s[rb*T + r][c] = sum over the chunks of row block rb of partial[chunk][target][r][c]
__global__ void k_hist_reduce(const int* __restrict__ chunk_ptr, const double* __restrict__ partial, int nrb,
                              int C2, double* __restrict__ s1, double* __restrict__ s2) {
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

}  // namespace

namespace mot {

void launch_history(mot_handle* h, const TaskList& tl, const double* tiles, const double* ring, const double* win,
                    const double* kry, int mode, long long step_i, double* out_s1, double* out_s2,
                    cudaStream_t s) {
    const int C2 = 2 * h->B;
    if (tl.nchunks > 0) {
        size_t smem = sizeof(double) * (T * (T + 1) + T * C2);
        const bool timed = h->opt.timing && mode == 0 && h->ev0 && step_i > h->K;
        if (timed) cudaEventRecord(h->ev0, s);
        k_hist_f64<<<tl.nchunks, NT, smem, s>>>(tl.tasks, tl.chunks, tiles, ring, win, kry, mode, step_i, h->R,
                                                h->npad, C2, h->d_colidx, h->d_partial);
        if (timed) {
            cudaEventRecord(h->ev1, s);
            h->ev_pending = true;
        }
        h->launches++;
    }
    k_hist_reduce<<<h->nrb, 256, 0, s>>>(tl.chunk_ptr, h->d_partial, h->nrb, C2, out_s1, out_s2);
    h->launches++;
}

}  // namespace mot
