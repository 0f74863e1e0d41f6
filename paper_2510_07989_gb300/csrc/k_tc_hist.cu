// History contraction of the mixed MOT path on the 5th-generation tensor cores
// (tcgen05 + TMEM), sm_100 family.
//
// The contraction is the lag sum of Eq. (MOT) in product form,
//   s1 = sum_k (A_k l_{i-k} + A^_k s_{i-k}),  s2 = sum_k (A~_k l_{i-k} + A_k s_{i-k}),
// stored as 32 x 32 tiles (row block x distance-sorted column block of that
// row block). One task multiplies one tile by the 32 coefficient rows it
// touches, for all 2B right-hand-side columns. On the tensor core a task is
// D[m][n] += sum_k P[m][k] X[n][k] with M = 128 (columns of the coefficient
// panel), N = 32 (tile rows), K = 32 (tile columns). A batch of B < 64 waves
// (B a multiple of 8) fills the first 2B of the 128 MMA rows; the others are
// never copied nor read back, and every column is computed as for B = 64.
//
// Every coefficient panel multiplies two tiles, one per output (s1, s2); a
// task gathers the panel once and multiplies both (the missing one is a zero
// tile).
//
// Precision: both operands are split into three bf16 slices, x = x0 + x1 + x2
// (each slice the round-to-nearest residual of the previous ones; the products
// of two bf16 values are exact in the FP32 accumulator). With Y, Z the tiles
// of s1 and s2, the six tile slices are stacked along N as [Y0 Z0 Y1 Z1 Y2 Z2]
// (32 rows each), so per K-half the tensor core runs
//   P0 x [Y0 Z0 Y1 Z1 Y2 Z2] (N = 192) into TMEM columns [0, 192),
//   P1 x [Y0 Z0 Y1 Z1]       (N = 128) into columns [64, 192),
//   P2 x [Y0 Z0]             (N = 64)  into columns [128, 192):
// columns [0, 64) hold only P0 Y0 | P0 Z0, [64, 128) the terms of relative
// size 2^-8, [128, 192) those of size 2^-16; per output the three blocks sum
// to P Y - (P1 Y2 + P2 Y1 + P2 Y2), a relative truncation of about 2^-26.
// Three MMAs per K-half, six per task: fewer, wider MMAs than one per
// (slice, slice) pair, since every instruction costs the single issuing
// thread the same whatever its N.
// The tensor core's FP32 accumulation rounds once per MMA at the scale of the
// accumulator, so the large block sees only two additions per task; after
// FGROUP tasks the epilogue warps fold the buffer into a compensated FP32 pair
// (TwoSum) per output element, so the sum over the thousands of tiles of a
// chunk carries no FP32 rounding growth. FP64 is not used in the loop: GB300
// issues about two FP64 operations per clock per SM.
//
// Coefficients: the ring keeps only the bf16 slices of l_j and s_j, columns
// [u | v]. The three forms a tile multiplies -- [eta u, v / eta],
// [eta' u, v / eta'] and [-v, u] -- are a per-column scale of the product
// (applied by the epilogue to a buffer that holds tasks of one form only) and,
// for the last, a swap of the two 64-column halves, done by the gather
// addresses. The windowed sums of the constant K~ tail are kept in their
// [-v, u] form and taken as they are.
//
// Data movement per task: the two tiles' three bf16 slices each, split once at
// set-up and stored in the swizzled B layout (2 KB per slice, contiguous), by
// six bulk copies (cp.async.bulk) whose bytes are added to the transaction
// count of the stage's FULL barrier; the coefficient rows, a gather through the
// row block's column order, by 16-byte cp.async copies that place every
// 16-byte piece straight into the swizzled MN-major A layout, each copying
// thread arriving on the same FULL barrier once its copies have landed.
// A pipeline stage holds the operands of TP = 1 or 2 tasks behind one FULL /
// EMPTY barrier pair: the producers wait and arrive once per stage, the MMA
// thread waits once and commits once per stage, so two tasks per stage halve
// the barrier hand-offs (NS stages: 4 or 5 of one task, 2 or 3 of two).
//
// Warp roles (224 threads with four epilogue warps, 352 with eight; one CTA
// per SM):
//   warps 0-1  gather: coefficient rows by cp.async (each lane's arrival fires
//              on completion of its copies, so the warps never wait for them)
//              and the tile copies
//   warp  2    TMEM allocation; lane 0 issues the MMAs
//   warps 3-6  epilogue (TMEM -> registers, compensated sums on packed FP32
//   (or 3-10)  pairs, partial results)
// Arrivals on a barrier are shared-memory atomics on one word: the epilogue
// warps arrive once per warp, after a warp-level sync.
// Every mbarrier wait is bounded in time; a wait that runs out raises the
// CTA's abort flag and the global error word, every role stops issuing work,
// copies in flight are waited for, and TMEM is released before the CTA exits.
#include <cuda_bf16.h>

#include <algorithm>

#include "mot_internal.h"
#include "tc_ptx.h"

using namespace tcx;

namespace {

constexpr int T = MOT_TILE;                 // 32
constexpr int TC_M = 128;                   // 2B columns per coefficient panel
constexpr int NB = 2;                       // TMEM accumulator buffers
constexpr int BUFCOLS = 192;                // TMEM columns per buffer (three magnitudes x two outputs x 32)
constexpr int TMEM_COLS = 512;              // allocation (power of two >= NB * BUFCOLS)
constexpr int FGROUP = 2;                   // tasks per TMEM accumulation
constexpr int A_SLICE = TC_M * T * 2;       // 8192 bytes: one bf16 slice of a 128 x 32 panel
constexpr int B_SLICE = T * T * 2;          // 2048 bytes: one bf16 slice of a tile
constexpr int STAGE_A = 3 * A_SLICE;        // 24576
constexpr int STAGE_B = 6 * B_SLICE;        // 12288: both tiles' slices, ordered X0 hi, X1 hi, X0 mid, X1 mid, X0 lo, X1 lo
constexpr int STAGE = STAGE_A + STAGE_B;    // 36864
constexpr int NPROD = 64;
// threads of a CTA with EW epilogue warps: warps 0-1 gather, 2 MMA, 3 .. 2 + EW
// epilogue (EW = 4: each warp folds both outputs of its TMEM lane quarter;
// EW = 8: two warps per quarter, one output each)
template <int EW>
__host__ __device__ constexpr int tc_threads() { return NPROD + 32 + 32 * EW; }
constexpr int TC_CHUNK = MOT_TC_CHUNK;      // tasks per CTA (staged in shared memory)
constexpr size_t TC_SMEM_MAX = 227 * 1024;

static_assert(NB * BUFCOLS <= TMEM_COLS, "TMEM buffers exceed the allocation");
static_assert(STAGE % 1024 == 0, "stage alignment");

// Shared-memory matrix descriptors (tcgen05 format: start >> 4, LBO >> 4,
// SBO >> 4, version 1 at bit 46, layout type at bits 61-63).
//
// A, the coefficient panel, MN-major with the 128-byte swizzle: atoms of 64
// columns (128 bytes) x 8 lag rows (1 KB), the 16-byte chunk c of row r stored
// at chunk position c ^ (r & 7); LBO = 4096 bytes between the two 64-column
// halves, SBO = 1024 bytes between groups of 8 rows along K.
__device__ __forceinline__ uint64_t desc_a_sw128(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(4096 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           (1ull << 46) | (2ull << 61);
}
// B, the tile slices: K-major with the 64-byte swizzle (desc_kmajor_sw64,
// sw64_chunk of the shared header).
// byte offset of the 16-byte chunk (m >> 3) of lag row k in an A slice
__host__ __device__ __forceinline__ uint32_t a_chunk(int k, int mg) {
    return (uint32_t)((mg >> 3) * 4096 + (k >> 3) * 1024 + (k & 7) * 128 + (((mg & 7) ^ (k & 7)) << 4));
}
// Instruction descriptor, kind::f16: FP32 accumulator, bf16 A and B, A
// MN-major (the coefficient panel, M contiguous), B K-major (the tile), M = 128.
__host__ __device__ constexpr uint32_t idesc_bf16(int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

__device__ __forceinline__ void split3(float x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
    a = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(a);  // exact
    b = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(b);  // exact
    c = __float2bfloat16_rn(r2);
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// Packed FP32 pairs: sm_100-family SMs issue one add, multiply or fma for
// two FP32 lanes (same IEEE round-to-nearest result per lane), which halves
// the instructions of the epilogue's compensated sums.
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as fma(b, -1, a): the product is exact, so one rounding as for a - b
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// s + c += v with the rounding error of s + v kept in c (Knuth's TwoSum), on
// both lanes of a pair
__device__ __forceinline__ void two_sum2(float2& s, float2& c, float2 v) {
    const float2 t = f2add(s, v);
    const float2 bp = f2sub(t, s);
    const float2 e = f2add(f2sub(s, f2sub(t, bp)), f2sub(v, bp));
    s = t;
    c = f2add(c, e);
}
__device__ __forceinline__ float2 pair_of(const float (&v)[32], int n) { return make_float2(v[2 * n], v[2 * n + 1]); }

__device__ __forceinline__ void producer_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// Merged task of the tensor-core list: x, y = tiles of s1 and s2 (the zero
// tile if absent), z = cb | k << 16 | (part | variant << 2) << 26.
__device__ __forceinline__ int pk_cb(uint4 d) { return (int)(d.z & 0xFFFFu); }
__device__ __forceinline__ int pk_k(uint4 d) { return (int)((d.z >> 16) & 0x3FFu); }
__device__ __forceinline__ int pk_code(uint4 d) { return (int)(d.z >> 26); }

// Coefficient transform of a task: its variant for l and s, 3 for the
// windowed sums (used as stored).
__device__ __forceinline__ int task_xform(int code) { return (code & 3) == 2 ? 3 : (code >> 2) & 3; }

// NS pipeline stages of TP tasks each (one FULL / EMPTY barrier pair per stage).
template <int NS, bool BULK, int TP>
struct TcLayout {
    // the gathered form stages the row block's column order in shared memory,
    // except with three stages of two tasks (no room left): it then reads it
    // through L1
    static constexpr bool SCOL = !BULK && (TP == 1 || NS == 2);
    static constexpr int NBARS = 2 * NS + 2 * NB + 1;  // + one barrier for the final MMA drain
    static constexpr size_t BARS = (size_t)NS * TP * STAGE;
    static constexpr size_t SLOT = BARS + ((8 * NBARS + 15) / 16) * 16;  // TMEM address, abort flag, issued count
    static constexpr size_t DESC = SLOT + 16;  // the chunk's packed tasks (uint4), cap of them
    // then (SCOL) the column order of the row block (uint16)
    static size_t bytes(int npad, int cap) {
        return DESC + 16 * (size_t)cap + (SCOL ? (((size_t)npad * 2 + 15) / 16) * 16 : 0) + 1024;
    }
    static_assert(BARS % 1024 == 0 && SLOT % 16 == 0 && DESC % 16 == 0,
                  "shared-memory regions must keep their alignment (uint4 task loads)");
};

// Element offset, in a blocked panel of the bulk form, of column m (0..127:
// half m >> 6, column m & 63 of the half) of coefficient row r of a 32-row
// block: each block is 8 KB, already in the MN-major 128-byte-swizzled layout
// of the MMA's A operand (a_chunk), so one bulk copy places it in shared memory.
__host__ __device__ __forceinline__ uint32_t blk_elem(int r, int m) {
    return (a_chunk(r, m >> 3) >> 1) + (uint32_t)(m & 7);
}

// BULK = false (gathered form): the columns of a row block are sorted by their
// distance from the block, and a panel's 32 coefficient rows are gathered from
// the ring ([npad][2B] per slice) by 16-byte cp.async copies of two warps,
// through the row block's column order staged in shared memory.
// BULK = true (bulk form): columns in the global (Morton) order, so the panel
// of column block cb is ring rows [32 cb, 32 cb + 32); the ring is stored in
// 32-row blocks already swizzled ([nrb][8 KB] per slice, u in the first 64-column
// half, v in the second), and one thread moves a stage with bulk copies: per
// slice one 8 KB copy (or two 4 KB copies with the halves exchanged for
// [-v, u]) and the six 2 KB tile slices, all counted in bytes on FULL.
// One launch serves one or several scatterers (jobs): the launch's CTAs are
// the chunks of job 0, then those of job 1, ... (cend: one past a job's last
// CTA). Every job brings its own task list, tiles, ring, output and error word.
struct TcJob {
    const uint4* tasks;
    const HistChunk* chunks;
    const __nv_bfloat16* tiles16;
    const __nv_bfloat16* ring16;
    const __nv_bfloat16* win16;
    const int* colidx;
    double* partial;
    int* err;
    long long step_i;
    double eta, etap;
    int R, npad, C2, cend;
};
struct TcJobs {
    int njobs;
    TcJob job[MOT_TC_MAX_JOBS];
};

template <int NS, bool BULK, int EW, int TP>
__global__ void __launch_bounds__(tc_threads<EW>(), 1)
    k_hist_tc(const __grid_constant__ TcJobs jobs, int cap, int stall_task, unsigned long long stall_bound) {
    constexpr int TC_THREADS = tc_threads<EW>();
    using L = TcLayout<NS, BULK, TP>;
    constexpr uint32_t SSTAGE = TP * STAGE;  // bytes of one pipeline stage (TP task slots of STAGE bytes)
    int jb = 0;
    while (jb + 1 < jobs.njobs && (int)blockIdx.x >= jobs.job[jb].cend) jb++;
    const TcJob& J = jobs.job[jb];
    const int cta = (int)blockIdx.x - (jb ? jobs.job[jb - 1].cend : 0);  // chunk of this job
    const uint4* __restrict__ tasks = J.tasks;
    const __nv_bfloat16* __restrict__ tiles16 = J.tiles16;
    const __nv_bfloat16* __restrict__ ring16 = J.ring16;
    const __nv_bfloat16* __restrict__ win16 = J.win16;
    const int* __restrict__ colidx = J.colidx;
    double* __restrict__ partial = J.partial;
    int* __restrict__ err = J.err;
    const long long step_i = J.step_i;
    const int R = J.R, npad = J.npad, C2 = J.C2;
    const double eta = J.eta, etap = J.etap;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // swizzled operand atoms need 1 KB alignment: the launch adds 1 KB of slack
    unsigned char* smem = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sbase = su32(smem);
    const uint32_t bar0 = sbase + (uint32_t)L::BARS;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L::SLOT);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    int* issued_slot = reinterpret_cast<int*>(tmem_slot + 2);  // stages whose copies the producers issued
    uint4* sdesc = reinterpret_cast<uint4*>(smem + L::DESC);
    uint16_t* scol = reinterpret_cast<uint16_t*>(smem + L::DESC + 16 * (size_t)cap);
    // FULL: the coefficient rows (one arrival per copying thread, when its
    // cp.async copies have landed) and the tile slices (bytes of the bulk
    // copies, added to the barrier's transaction count) of a stage's tasks
    auto FULL = [&](int s) { return bar0 + 8u * s; };
    auto EMPTY = [&](int s) { return bar0 + 8u * (NS + s); };  // MMAs done with the stage
    auto ACCF = [&](int b) { return bar0 + 8u * (2 * NS + b); };
    auto ACCE = [&](int b) { return bar0 + 8u * (2 * NS + NB + b); };
    const uint32_t DRAIN = bar0 + 8u * (2 * NS + 2 * NB);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const HistChunk ch = J.chunks[cta];
    // failure test (stall_task >= 0): the first CTA withholds the copies and
    // arrivals of its stage stall_task, and every wait of that CTA gives up
    // after stall_bound ns, so the launch ends through the abort path
    const bool stall_cta = stall_task >= 0 && blockIdx.x == 0;
    const unsigned long long bound = stall_cta ? stall_bound : WAIT_NS;
    const int ntask = ch.count;  // <= cap

    // the chunk's task list and the row block's column order, staged once
    for (int i = tid; i < ntask; i += TC_THREADS) sdesc[i] = tasks[ch.first + i];
    if (L::SCOL)
        for (int p = tid; p < npad; p += TC_THREADS) scol[p] = (uint16_t)colidx[(size_t)ch.rb * npad + p];
    const int* __restrict__ gcol = colidx + (size_t)ch.rb * npad;  // the same order in global memory
    if (tid == 0) {
        for (int s = 0; s < NS; s++) {
            mbar_init(FULL(s), BULK ? 1 : NPROD);
            mbar_init(EMPTY(s), 1);
        }
        for (int b = 0; b < NB; b++) {
            mbar_init(ACCF(b), 1);
            mbar_init(ACCE(b), EW);
        }
        mbar_init(DRAIN, 1);
        *abort_flag = 0;
        *issued_slot = 0;
        fence_barrier_init();
    }
    if (warp == 2) {
        tmem_alloc(su32(tmem_slot), TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (BULK && warp < 2) {
        // ---------------- bulk producer: one thread moves every stage ----------------
        if (tid == 0) {
            const int slot_i = (int)(step_i % R);
            const size_t pslice = (size_t)npad * 128;  // elements of one slice of one ring part (all blocks)
            int v = 0;  // tasks that take part (lag within the march so far)
            int s = 0;
            for (int ti = 0; ti < ntask; ti++) {
                const uint4 d = sdesc[ti];
                const int cb = pk_cb(d), k = pk_k(d), code = pk_code(d);
                if (step_i - k < 1) continue;
                const int j = v / TP, u = v % TP;
                s = j % NS;
                v++;
                if (u == 0) {
                    if (!mbar_wait(EMPTY(s), ((uint32_t)(j / NS) & 1u) ^ 1u, abort_flag, err, 2, bound)) {
                        v = -1;
                        break;
                    }
                    *issued_slot = j + 1;
                }
                if (stall_cta && j == stall_task) continue;  // failure test: this stage is never filled
                mbar_add_tx(FULL(s), STAGE);  // every byte of the task, before the stage's one arrival
                const uint32_t adst = sbase + s * SSTAGE + u * STAGE;
#pragma unroll
                for (int q = 0; q < 3; q++) {
                    bulk_g2s(adst + STAGE_A + (2 * q) * B_SLICE, tiles16 + ((size_t)d.x * 3 + q) * (T * T), B_SLICE,
                             FULL(s));
                    bulk_g2s(adst + STAGE_A + (2 * q + 1) * B_SLICE, tiles16 + ((size_t)d.y * 3 + q) * (T * T),
                             B_SLICE, FULL(s));
                }
                const int part = code & 3, var = (code >> 2) & 3;
                const __nv_bfloat16* blk =
                    (part == 2 ? win16 + (size_t)k * 3 * pslice
                               : ring16 + (((size_t)(slot_i - k + (slot_i < k ? R : 0)) * 2 + part) * 3) * pslice) +
                    (size_t)cb * (T * 128);
                if (part != 2 && var == 2) {  // [-v, u]: the v half first
#pragma unroll
                    for (int q = 0; q < 3; q++) {
                        bulk_g2s(adst + q * A_SLICE, blk + q * pslice + T * 64, A_SLICE / 2, FULL(s));
                        bulk_g2s(adst + q * A_SLICE + A_SLICE / 2, blk + q * pslice, A_SLICE / 2, FULL(s));
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 3; q++) bulk_g2s(adst + q * A_SLICE, blk + q * pslice, A_SLICE, FULL(s));
                }
                if (u == TP - 1) mbar_arrive(FULL(s));  // the stage is complete
            }
            // a last stage with fewer than TP tasks
            if (v > 0 && v % TP != 0 && !(stall_cta && (v - 1) / TP == stall_task)) mbar_arrive(FULL(s));
        }
    } else if (!BULK && warp < 2) {
        // ---------------- gather: coefficient rows and the tile copy ----------------
        const int t = tid;
        const int l8 = lane & 7, l3 = lane >> 3;
        const int slot_i = (int)(step_i % R);  // ring slot of step i; lag k (< R) is slot_i - k mod R
        // this lane's 16-byte pieces: slices q = 0..2, row groups ro, column quads mq of
        // its warp's half (mq = 2 warp + 0/1); destination offsets do not depend on the task
        uint32_t dofs[4][2];
#pragma unroll
        for (int ro = 0; ro < 4; ro++)
#pragma unroll
            for (int h = 0; h < 2; h++) dofs[ro][h] = a_chunk(ro * 8 + l8, (2 * warp + h) * 4 + l3);
        const size_t pstride = (size_t)npad * C2;  // elements of one bf16 slice of one panel
        // 16-byte pieces per coefficient row (C2 / 8); a batch below 64 waves
        // leaves the panel's upper columns uncopied (their TMEM lanes are never
        // read). Source offsets of this lane's two pieces, as stored and with
        // the u and v halves exchanged ([-v, u]), fixed for the whole chunk.
        const int nch = C2 >> 3;
        int soff0[2], soff1[2];
        bool has[2];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int mg = (2 * warp + h) * 4 + l3;
            has[h] = mg < nch;
            const int sw = mg + (nch >> 1) < nch ? mg + (nch >> 1) : mg + (nch >> 1) - nch;
            soff0[h] = mg * 8;
            soff1[h] = sw * 8;
        }
        int v = 0;  // tasks that take part
        int s = 0;
        for (int ti = 0; ti < ntask; ti++) {
            const uint4 d = sdesc[ti];
            const int cb = pk_cb(d), k = pk_k(d), code = pk_code(d);
            if (step_i - k < 1) continue;
            const int j = v / TP, u = v % TP;
            s = j % NS;
            v++;
            if (u == 0) {
                if (!mbar_wait(EMPTY(s), ((uint32_t)(j / NS) & 1u) ^ 1u, abort_flag, err, 2, bound)) {
                    v = -1;
                    break;
                }
                if (t == 0) *issued_slot = j + 1;
            }
            if (stall_cta && j == stall_task) continue;  // failure test: this stage is never filled
            const uint32_t adst = sbase + s * SSTAGE + u * STAGE;
            if (t == 0) {  // slices in the order Y0 Z0 Y1 Z1 Y2 Z2; bytes added before this thread's arrival
                mbar_add_tx(FULL(s), STAGE_B);
#pragma unroll
                for (int q = 0; q < 3; q++) {
                    bulk_g2s(adst + STAGE_A + (2 * q) * B_SLICE, tiles16 + ((size_t)d.x * 3 + q) * (T * T), B_SLICE,
                             FULL(s));
                    bulk_g2s(adst + STAGE_A + (2 * q + 1) * B_SLICE, tiles16 + ((size_t)d.y * 3 + q) * (T * T),
                             B_SLICE, FULL(s));
                }
            }
            const int part = code & 3, var = (code >> 2) & 3;
            const __nv_bfloat16* pan = part == 2 ? win16 + (size_t)k * 3 * pstride
                                                 : ring16 + (((size_t)(slot_i - k + (slot_i < k ? R : 0)) * 2 + part) * 3) * pstride;
            const int swap = (part != 2 && var == 2) ? 1 : 0;  // [-v, u]: the u and v halves exchanged
#pragma unroll
            for (int ro = 0; ro < 4; ro++) {
                const int c = cb * T + ro * 8 + l8;
                const __nv_bfloat16* row = pan + (size_t)(L::SCOL ? (int)scol[c] : __ldg(gcol + c)) * C2;
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    if (!has[h]) continue;
                    const __nv_bfloat16* src = row + (swap ? soff1[h] : soff0[h]);
#pragma unroll
                    for (int q = 0; q < 3; q++) cp_async16(adst + q * A_SLICE + dofs[ro][h], src + (size_t)q * pstride);
                }
            }
            // this thread's arrival on the stage fires when its copies have landed
            if (u == TP - 1) cp_async_arrive_noinc(FULL(s));
        }
        // a last stage with fewer than TP tasks
        if (v > 0 && v % TP != 0 && !(stall_cta && (v - 1) / TP == stall_task)) cp_async_arrive_noinc(FULL(s));
        cp_async_wait_all();  // this thread's row copies have landed
    } else if (warp == 2) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            int v = 0, g = -1, ing = 0, cur = -1, s = 0;
            uint32_t dcol = 0;
            for (int ti = 0; ti < ntask; ti++) {
                const uint4 d = sdesc[ti];
                if (step_i - pk_k(d) < 1) continue;
                const int key = task_xform(pk_code(d));  // a buffer holds tasks of one coefficient transform
                if (g < 0 || key != cur || ing == FGROUP) {
                    if (g >= 0) tc_commit(ACCF(g % NB));
                    g++;
                    ing = 0;
                    cur = key;
                    const int b = g % NB;
                    if (!mbar_wait(ACCE(b), ((uint32_t)(g / NB) & 1u) ^ 1u, abort_flag, err, 3, bound)) break;
                    tc_fence_after();
                    dcol = tmem + (uint32_t)(b * BUFCOLS);
                }
                const int j = v / TP, u = v % TP;
                s = j % NS;
                if (u == 0) {
                    if (!mbar_wait(FULL(s), (uint32_t)(j / NS) & 1u, abort_flag, err, 4, bound)) break;
                    if (!BULK) fence_proxy_async();  // coefficient rows written by cp.async (generic proxy)
                    tc_fence_after();
                }
                const uint32_t a0 = sbase + s * SSTAGE + u * STAGE, b0 = a0 + STAGE_A;
                // K-half kk: A rows 16 kk .. 16 kk + 15 (two 1 KB row groups),
                // B columns 16 kk .. (32 bytes into each 64-byte row)
#pragma unroll
                for (int kk = 0; kk < 2; kk++) {
                    const uint64_t bd = desc_kmajor_sw64(b0 + kk * 32);
                    mma_bf16(dcol, desc_a_sw128(a0 + kk * 2048), bd, idesc_bf16(192), (ing > 0 || kk > 0) ? 1u : 0u);
                    mma_bf16(dcol + 64, desc_a_sw128(a0 + A_SLICE + kk * 2048), bd, idesc_bf16(128), 1u);
                    mma_bf16(dcol + 128, desc_a_sw128(a0 + 2 * A_SLICE + kk * 2048), bd, idesc_bf16(64), 1u);
                }
                if (u == TP - 1) tc_commit(EMPTY(s));  // the stage's tasks are done with its buffers
                ing++;
                v++;
            }
            if (v % TP != 0) tc_commit(EMPTY(s));  // a last stage with fewer than TP tasks
            // the last (or interrupted) group: its commit also tells the
            // epilogue that every MMA issued by this thread has completed
            if (g >= 0) tc_commit(ACCF(g % NB));
            // TMEM is released only after every MMA of this CTA has completed
            tc_commit(DRAIN);
            mbar_wait_drain(DRAIN, 0, bound);
        }
        __syncwarp();
    } else {
        // ---------------- epilogue ----------------
        const int quarter = warp & 3;  // TMEM lanes [32 quarter, 32 quarter + 32)
        const int m = quarter * 32 + lane;
        const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
        // outputs this warp folds: both (EW = 4), or one (EW = 8: warps 3-6 s1, 7-10 s2)
        constexpr int NO = EW == 8 ? 1 : 2;
        const int o0 = EW == 8 ? (warp - 3) >> 2 : 0;
        float2 hs[NO][16], hc[NO][16];  // compensated sums, tile rows 2n and 2n + 1 in a pair
#pragma unroll
        for (int o = 0; o < NO; o++)
#pragma unroll
            for (int n = 0; n < 16; n++) hs[o][n] = hc[o][n] = make_float2(0.f, 0.f);
        // per-column scale of each coefficient transform. Gathered form: panel
        // column m is u of wave m (m < B) or v of wave m - B. Bulk form: u of
        // wave m & 63 in the first half (m < 64), v in the second.
        const int Bw = C2 / 2;
        const bool ucol = BULK ? m < 64 : m < Bw;
        const int ocol = BULK ? ((m & 63) < Bw ? (m >> 6) * Bw + (m & 63) : -1) : (m < C2 ? m : -1);
        const float xs0 = ucol ? (float)eta : (float)(1.0 / eta), xs1 = ucol ? (float)etap : (float)(1.0 / etap),
                    xs2 = ucol ? -1.f : 1.f;
        // folds the 32 columns at col into sums o; the last fold of a buffer
        // releases it (one arrival per epilogue warp)
        auto fold = [&](uint32_t col, float c, int o, bool release, int b) {
            float va[32], vb[32];
            const float2 cc = make_float2(c, c);
            if constexpr (EW == 8) {
                // one output per warp: the three blocks in one round trip of
                // TMEM loads, then the buffer is released before the arithmetic
                float vl[32];
                tmem_ld32(col + 64, va);   // terms of relative size 2^-8
                tmem_ld32(col + 128, vb);  // and 2^-16
                tmem_ld32(col, vl);        // the leading products
                tmem_wait_ld();
                if (release) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(ACCE(b));
                }
#pragma unroll
                for (int n = 0; n < 16; n++)
                    hc[o][n] = f2fma(cc, pair_of(vb, n), f2fma(cc, pair_of(va, n), hc[o][n]));
#pragma unroll
                for (int n = 0; n < 16; n++) two_sum2(hs[o][n], hc[o][n], f2mul(cc, pair_of(vl, n)));
            } else {
                tmem_ld32(col + 64, va);   // terms of relative size 2^-8
                tmem_ld32(col + 128, vb);  // and 2^-16
                tmem_wait_ld();
#pragma unroll
                for (int n = 0; n < 16; n++)
                    hc[o][n] = f2fma(cc, pair_of(vb, n), f2fma(cc, pair_of(va, n), hc[o][n]));
                tmem_ld32(col, va);  // the leading products
                tmem_wait_ld();
                if (release) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(ACCE(b));
                }
#pragma unroll
                for (int n = 0; n < 16; n++) two_sum2(hs[o][n], hc[o][n], f2mul(cc, pair_of(va, n)));
            }
        };
        auto drain = [&](int gg, int key) -> bool {
            const int b = gg % NB;
            if (!mbar_wait(ACCF(b), (uint32_t)(gg / NB) & 1u, abort_flag, err, 5, bound)) return false;
            tc_fence_after();
            __syncwarp();
            const float c = key == 0 ? xs0 : key == 1 ? xs1 : key == 2 ? xs2 : 1.f;
            const uint32_t col = tl + (uint32_t)(b * BUFCOLS);
#pragma unroll
            for (int o = 0; o < NO; o++) fold(col + 32 * (o0 + o), c, o, o == NO - 1, b);
            return true;
        };
        int g = -1, ing = 0, cur = -1;
        bool ok = true;
        for (int ti = 0; ti < ntask && ok; ti++) {
            const uint4 d = sdesc[ti];
            if (step_i - pk_k(d) < 1) continue;
            const int key = task_xform(pk_code(d));
            if (g < 0 || key != cur || ing == FGROUP) {
                if (g >= 0 && !drain(g, cur)) {
                    ok = false;
                    break;
                }
                g++;
                ing = 0;
                cur = key;
            }
            ing++;
        }
        if (ok && g >= 0) drain(g, cur);
        if (ocol >= 0) {
#pragma unroll
            for (int o = 0; o < NO; o++) {
                double* p = partial + ((size_t)cta * 2 + o0 + o) * T * C2 + ocol;
#pragma unroll
                for (int n = 0; n < 16; n++) {
                    p[(size_t)(2 * n) * C2] = (double)hs[o][n].x + (double)hc[o][n].x;
                    p[(size_t)(2 * n + 1) * C2] = (double)hs[o][n].y + (double)hc[o][n].y;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 2) {
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
    // After an abort (every role has stopped: the flag is final here), tile
    // copies of stages the MMA thread never consumed may still be in flight:
    // wait (bounded) for the last NS issued stages before the CTA's shared
    // memory is released.
    if (tid == 0 && *abort_flag) {
        const int issued = *issued_slot;
        for (int jj = issued > NS ? issued - NS : 0; jj < issued; jj++)
            mbar_wait_drain(FULL(jj % NS), (uint32_t)(jj / NS) & 1u, bound);
    }
}

// src: npanels panels of n doubles; dst: npanels x 3 bf16 slices of n values.
// Blocked (bulk-form) panels: n = npad x 2B values per panel become three
// slices of npad x 128 bf16 each, in 32-row blocks of blk_elem layout (the
// first B columns of a row in the first half, the next B in the second; the
// other columns stay as allocated, zero).
__global__ void k_split3(size_t n, int npanels, int C2, int blocked, const double* __restrict__ src,
                         __nv_bfloat16* __restrict__ dst) {
    const size_t total = n * (size_t)npanels;
    const size_t ns = blocked ? n / C2 * 128 : n;  // elements of one slice
    const int B = C2 / 2;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t p = i / n, r = i - p * n;
        const double x = src[i];
        const __nv_bfloat16 a = __double2bfloat16(x);
        const double r1 = x - (double)__bfloat162float(a);
        const __nv_bfloat16 b = __double2bfloat16(r1);
        const double r2 = r1 - (double)__bfloat162float(b);
        const __nv_bfloat16 c = __double2bfloat16(r2);
        size_t e = r;
        if (blocked) {
            const size_t row = r / C2;
            const int m = (int)(r - row * C2);
            const int mm = m < B ? m : 64 + m - B;
            e = (row >> 5) * (T * 128) + blk_elem((int)(row & 31), mm);
        }
        __nv_bfloat16* d = dst + p * 3 * ns + e;
        d[0] = a;
        d[ns] = b;
        d[2 * ns] = c;
    }
}

// Tiles for the tensor-core kernel: each FP32 32 x 32 tile as three bf16
// slices, already in the K-major 64-byte-swizzled layout of the MMA's B
// operand (6 KB per tile, copied to shared memory as is). The split is exact:
// hi + mid + lo reproduces the FP32 value.
__global__ void k_split_tiles(long long ntiles, const float* __restrict__ src, __nv_bfloat16* __restrict__ dst) {
    const long long total = ntiles * T * 4;  // (tile, row, 8-column group)
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long t = i / (T * 4);
        const int r = (int)(i - t * T * 4) >> 2, kc = (int)(i & 3);
        const float* x = src + (size_t)t * T * T + r * T + kc * 8;
        __nv_bfloat16 a[8], b[8], c[8];
#pragma unroll
        for (int e = 0; e < 8; e++) split3(x[e], a[e], b[e], c[e]);
        unsigned char* d = reinterpret_cast<unsigned char*>(dst + (size_t)t * 3 * T * T) + sw64_chunk(r, kc);
        *reinterpret_cast<uint4*>(d) = make_uint4(pack2(a[0], a[1]), pack2(a[2], a[3]), pack2(a[4], a[5]), pack2(a[6], a[7]));
        *reinterpret_cast<uint4*>(d + B_SLICE) =
            make_uint4(pack2(b[0], b[1]), pack2(b[2], b[3]), pack2(b[4], b[5]), pack2(b[6], b[7]));
        *reinterpret_cast<uint4*>(d + 2 * B_SLICE) =
            make_uint4(pack2(c[0], c[1]), pack2(c[2], c[3]), pack2(c[4], c[5]), pack2(c[6], c[7]));
    }
}

// bf16 slices of l and s of one ring slot, columns [u | v], from the FP64
// ring's [-v, u] variant of each part: dst [2 parts][3 slices][npad][2B]
// (gathered form), or [2 parts][3 slices][npad x 128] in blk_elem blocks, u in
// the first half and v in the second (bulk form).
__global__ void k_split_ring(int npad, int B, int blocked, const double* __restrict__ ring_slot,
                             __nv_bfloat16* __restrict__ dst) {
    const int C2 = 2 * B;
    const size_t ps = (size_t)npad * C2;                  // FP64 values of one part's variant
    const size_t ds = blocked ? (size_t)npad * 128 : ps;  // elements of one destination slice
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < 2 * ps; i += (size_t)gridDim.x * blockDim.x) {
        const int part = (int)(i / ps);
        const size_t r = (i - part * ps) / C2;
        const int m = (int)(i - part * ps - r * C2);
        const double* v2 = ring_slot + ((size_t)part * 3 + 2) * ps + r * C2;  // [-v, u]
        const double x = m < B ? v2[B + m] : -v2[m - B];
        const __nv_bfloat16 a = __double2bfloat16(x);
        const double r1 = x - (double)__bfloat162float(a);
        const __nv_bfloat16 b = __double2bfloat16(r1);
        const double r2 = r1 - (double)__bfloat162float(b);
        const size_t e = blocked ? (r >> 5) * (T * 128) + blk_elem((int)(r & 31), m < B ? m : 64 + m - B) : r * C2 + m;
        __nv_bfloat16* d = dst + (size_t)part * 3 * ds + e;
        d[0] = a;
        d[ds] = b;
        d[2 * ds] = __double2bfloat16(r2);
    }
}

// s1, s2 of row block rb = sum of the partial results of its chunks, in the
// order of the row block's chunk list.
__global__ void k_hist_reduce_idx(const int* __restrict__ rb_ptr, const int* __restrict__ rb_chunks,
                                  const double* __restrict__ partial, int C2, double* __restrict__ s1,
                                  double* __restrict__ s2) {
    const int rb = blockIdx.x;
    const int nout = T * C2;
    const int c0 = rb_ptr[rb], c1 = rb_ptr[rb + 1];
    for (int o = threadIdx.x; o < nout; o += blockDim.x) {
        double a = 0.0, b = 0.0;
        for (int ci = c0; ci < c1; ci++) {
            const size_t c = (size_t)rb_chunks[ci];
            a += partial[c * 2 * nout + o];
            b += partial[c * 2 * nout + nout + o];
        }
        s1[(size_t)rb * nout + o] = a;
        s2[(size_t)rb * nout + o] = b;
    }
}

}  // namespace

namespace mot {

void launch_split_tiles(mot_handle* h, cudaStream_t s) {
    const long long total = h->ntiles * T * 4;
    if (total == 0) return;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 32);
    k_split_tiles<<<blocks, 256, 0, s>>>(h->ntiles, h->d_tiles32, reinterpret_cast<__nv_bfloat16*>(h->d_tiles16));
    h->launches++;
}

void launch_split_ring(mot_handle* h, int slot, cudaStream_t s) {
    const size_t bv = (size_t)h->npad * 2 * h->B;
    const size_t slot16 = history_tc_ring_slot_elems(h);
    const int blocks = (int)std::min<size_t>((2 * bv + 255) / 256, 152 * 16);
    k_split_ring<<<blocks, 256, 0, s>>>(h->npad, h->B, h->tc_bulk ? 1 : 0, h->d_ring + (size_t)slot * 6 * bv,
                                        reinterpret_cast<__nv_bfloat16*>(h->d_ring16) + (size_t)slot * slot16);
    h->launches++;
}

size_t history_tc_ring_slot_elems(const mot_handle* h) {
    // 2 parts x 3 slices of npad x 2B (gathered form) or npad x 128 (bulk form)
    return (size_t)6 * h->npad * (h->tc_bulk ? 128 : 2 * h->B);
}


// Pipeline configurations of the history kernel: (stages, tasks per stage).
// Whether one fits in shared memory with `cap` staged tasks (and, for the
// gathered form with one task per stage, the row block's column order).
bool history_tc_config_fits(int npad, bool bulk, int cap, int ns, int tp) {
    if (npad > 65536) return false;
    size_t b = 0;
    if (tp == 1) {
        if (ns == 4) b = bulk ? TcLayout<4, true, 1>::bytes(npad, cap) : TcLayout<4, false, 1>::bytes(npad, cap);
        else if (ns == 5) b = bulk ? TcLayout<5, true, 1>::bytes(npad, cap) : TcLayout<5, false, 1>::bytes(npad, cap);
        else return false;
    } else if (tp == 2) {
        if (ns == 2) b = bulk ? TcLayout<2, true, 2>::bytes(npad, cap) : TcLayout<2, false, 2>::bytes(npad, cap);
        else if (ns == 3) b = bulk ? TcLayout<3, true, 2>::bytes(npad, cap) : TcLayout<3, false, 2>::bytes(npad, cap);
        else return false;
    } else {
        return false;
    }
    return b <= TC_SMEM_MAX;
}

// the default configuration: the deepest one-task pipeline that fits
int history_tc_stages(int npad, bool bulk, int cap) {
    if (history_tc_config_fits(npad, bulk, cap, 5, 1)) return 5;
    return history_tc_config_fits(npad, bulk, cap, 4, 1) ? 4 : 0;
}

bool history_tc_fits(int npad, bool bulk) { return history_tc_stages(npad, bulk, MOT_TC_CHUNK) > 0; }

void launch_split3(mot_handle* h, int npanels, const double* src, uint16_t* dst, cudaStream_t s) {
    const size_t n = (size_t)h->npad * 2 * h->B;
    const size_t total = n * (size_t)npanels;
    if (total == 0) return;
    const int blocks = (int)std::min<size_t>((total + 255) / 256, 152 * 16);
    k_split3<<<blocks, 256, 0, s>>>(n, npanels, 2 * h->B, h->tc_bulk ? 1 : 0, src, reinterpret_cast<__nv_bfloat16*>(dst));
    h->launches++;
}

namespace {

TcJob job_of(mot_handle* h, long long step_i) {
    TcJob j;
    j.tasks = h->hist_tc_list.packed;
    j.chunks = h->hist_tc_list.chunks;
    j.tiles16 = reinterpret_cast<const __nv_bfloat16*>(h->d_tiles16);
    j.ring16 = reinterpret_cast<const __nv_bfloat16*>(h->d_ring16);
    j.win16 = reinterpret_cast<const __nv_bfloat16*>(h->d_win16);
    j.colidx = h->d_colidx;
    j.partial = h->d_partial;
    j.err = h->d_cg_iters + 2;
    j.step_i = step_i;
    j.eta = h->eta;
    j.etap = h->etap;
    j.R = h->R;
    j.npad = h->npad;
    j.C2 = 2 * h->B;
    j.cend = 0;
    return j;
}

// One launch of the history kernel over jobs[0 .. njobs) (all of one form);
// the pipeline (stages x tasks per stage) is the first handle's tuned or set
// one when it fits in shared memory, else the deepest one-task pipeline that
// fits.
void launch_jobs(mot_handle* h0, TcJobs& jobs, int nctas, int max_npad, int cap, cudaStream_t s) {
    static std::atomic<unsigned long long> attr{0};
    once_per_device(attr, h0->dev, [] {
        const int mx = (int)TC_SMEM_MAX;
#define MOT_TC_ATTR(NSV, BV, EWV, TPV) \
    cudaFuncSetAttribute(k_hist_tc<NSV, BV, EWV, TPV>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx)
#define MOT_TC_ATTR_ALL(BV, EWV) \
    MOT_TC_ATTR(4, BV, EWV, 1);  \
    MOT_TC_ATTR(5, BV, EWV, 1);  \
    MOT_TC_ATTR(2, BV, EWV, 2);  \
    MOT_TC_ATTR(3, BV, EWV, 2)
        MOT_TC_ATTR_ALL(false, 4);
        MOT_TC_ATTR_ALL(false, 8);
        MOT_TC_ATTR_ALL(true, 4);
        MOT_TC_ATTR_ALL(true, 8);
#undef MOT_TC_ATTR_ALL
#undef MOT_TC_ATTR
    });
    // failure test of the bounded waits (mot_options.hist_stall_test), off by default
    const int stall = h0->opt.hist_stall_test > 0 ? h0->opt.hist_stall_test - 1 : -1;
    // the handles' tuned configuration if it fits, else the deepest one-task pipeline
    int ns = h0->tc_stages, tp = h0->tc_tps;
    if (ns <= 0 || !history_tc_config_fits(max_npad, h0->tc_bulk, cap, ns, tp)) {
        ns = history_tc_stages(max_npad, h0->tc_bulk, cap);
        tp = 1;
    }
    const bool e8 = h0->tc_epi == 8;
#define MOT_TC_LAUNCH(NSV, BV, EWV, TPV)                                                                         \
    k_hist_tc<NSV, BV, EWV, TPV><<<nctas, tc_threads<EWV>(), TcLayout<NSV, BV, TPV>::bytes(max_npad, cap), s>>>( \
        jobs, cap, stall, 1000000ull)
#define MOT_TC_LAUNCH_CFG(BV, EWV)                        \
    if (tp == 2 && ns == 3) MOT_TC_LAUNCH(3, BV, EWV, 2); \
    else if (tp == 2) MOT_TC_LAUNCH(2, BV, EWV, 2);       \
    else if (ns == 5) MOT_TC_LAUNCH(5, BV, EWV, 1);       \
    else MOT_TC_LAUNCH(4, BV, EWV, 1)
    if (h0->tc_bulk) {
        if (e8) MOT_TC_LAUNCH_CFG(true, 8);
        else MOT_TC_LAUNCH_CFG(true, 4);
    } else {
        if (e8) MOT_TC_LAUNCH_CFG(false, 8);
        else MOT_TC_LAUNCH_CFG(false, 4);
    }
#undef MOT_TC_LAUNCH_CFG
#undef MOT_TC_LAUNCH
    h0->launches++;
}

}  // namespace

void launch_history_tc(mot_handle* h, const TaskList& tl, long long step_i, double* out_s1, double* out_s2,
                       cudaStream_t s) {
    const int C2 = 2 * h->B;
    if (tl.nchunks > 0) {
        const bool timed = h->opt.timing && h->ev0 && step_i > h->K;
        if (timed) cudaEventRecord(h->ev0, s);
        TcJobs jobs;
        jobs.njobs = 1;
        jobs.job[0] = job_of(h, step_i);
        jobs.job[0].tasks = tl.packed;
        jobs.job[0].chunks = tl.chunks;
        jobs.job[0].cend = tl.nchunks;
        launch_jobs(h, jobs, tl.nchunks, h->npad, tl.cap, s);
        h->tc_launches++;
        if (timed) {
            cudaEventRecord(h->ev1, s);
            h->ev_pending = true;
        }
    }
    k_hist_reduce_idx<<<h->nrb, 256, 0, s>>>(tl.rb_ptr, tl.rb_chunks, h->d_partial, C2, out_s1, out_s2);
    h->launches++;
}

// The history of n scatterers (all on the tensor-core path, one form) in one
// launch of the history kernel: step i of handle k is hs[k]->step + 1; the
// chunk sums of every handle are then reduced into s1[k], s2[k]. All on
// stream s. Returns the launch's duration in ms when `timed` (events on s).
float launch_history_tc_many(mot_handle* const* hs, int n, double* const* s1, double* const* s2, cudaStream_t s,
                             bool timed) {
    TcJobs jobs;
    jobs.njobs = n;
    int nctas = 0, max_npad = 0, cap = 1;
    for (int k = 0; k < n; k++) {
        mot_handle* h = hs[k];
        jobs.job[k] = job_of(h, h->step + 1);
        nctas += h->hist_tc_list.nchunks;
        jobs.job[k].cend = nctas;
        max_npad = std::max(max_npad, h->npad);
        cap = std::max(cap, h->hist_tc_list.cap);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (timed && nctas > 0) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, s);
    }
    if (nctas > 0) {
        launch_jobs(hs[0], jobs, nctas, max_npad, cap, s);
        for (int k = 0; k < n; k++) hs[k]->tc_launches++;
    }
    if (e1) cudaEventRecord(e1, s);
    for (int k = 0; k < n; k++) {
        mot_handle* h = hs[k];
        k_hist_reduce_idx<<<h->nrb, 256, 0, s>>>(h->hist_tc_list.rb_ptr, h->hist_tc_list.rb_chunks, h->d_partial,
                                                 2 * h->B, s1[k], s2[k]);
        h->launches++;
    }
    float ms = 0.f;
    if (e1) {
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    return ms;
}

}  // namespace mot
