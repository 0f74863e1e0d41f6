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
//
// Warp roles (224 threads, one CTA per SM):
//   warps 0-1  gather: coefficient rows by cp.async (each lane's arrival fires
//              on completion of its copies, so the warps never wait for them)
//              and the tile copies
//   warp  2    TMEM allocation; lane 0 issues the MMAs
//   warps 3-6  epilogue (TMEM -> registers, compensated sums, partial results)
// Arrivals on a barrier are shared-memory atomics on one word: the epilogue
// warps arrive once per warp, after a warp-level sync.
// Every mbarrier wait is bounded in time; a wait that runs out raises the
// CTA's abort flag and the global error word, every role stops issuing work,
// copies in flight are waited for, and TMEM is released before the CTA exits.
#include <cuda_bf16.h>

#include <algorithm>

#include "mot_internal.h"

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
constexpr int NPROD = 64, NEPI = 128;
constexpr int TC_THREADS = NPROD + 32 + NEPI;  // 224: warps 0-1 gather, 2 MMA, 3-6 epilogue
constexpr int TC_CHUNK = MOT_TC_CHUNK;      // tasks per CTA (staged in shared memory)
constexpr size_t TC_SMEM_MAX = 227 * 1024;
constexpr unsigned long long WAIT_NS = 2000000000ull;  // bound of every wait (2 s)

static_assert(NB * BUFCOLS <= TMEM_COLS, "TMEM buffers exceed the allocation");
static_assert(STAGE % 1024 == 0, "stage alignment");

// ---- PTX wrappers -----------------------------------------------------------
__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Raise the barrier's expected transaction count without arriving.
__device__ __forceinline__ void mbar_add_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of the given parity. Returns false when the CTA
// was told to abort or when the bound ran out (then it raises the abort flag
// and records `code` in the global error word). The slow path (time bound,
// abort flag) is out of line and entered only after many failed tries, so the
// common case costs no call.
__device__ __noinline__ bool mbar_wait_slow(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* err,
                                            int code) {
    const unsigned long long t0 = gtimer();
    for (;;) {
        for (int i = 0; i < 64; i++)
            if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > WAIT_NS) {
            *abort_flag = 1;
            atomicExch(err, code);
            return false;
        }
    }
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* err,
                                          int code) {
#pragma unroll 1
    for (int i = 0; i < 4096; i++)
        if (mbar_try(bar, parity)) return true;
    return mbar_wait_slow(bar, parity, abort_flag, err, code);
}

// Wait used while shutting down after an abort: bounded, ignores the flag.
__device__ __noinline__ void mbar_wait_drain(uint32_t bar, uint32_t parity) {
    const unsigned long long t0 = gtimer();
    while (!mbar_try(bar, parity))
        if (gtimer() - t0 > WAIT_NS) return;
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
// Arrive on the mbarrier once all prior cp.async copies of this thread have
// landed (the arrival is counted in the barrier's expected count).
__device__ __forceinline__ void cp_async_arrive_noinc(uint32_t bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] x B[smem]^T, bf16 inputs, FP32 accumulation.
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive once on the mbarrier when all tcgen05 operations issued so far by
// this thread have completed.
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 32 lanes x 32 consecutive columns of 32 bits: thread t of the warp gets
// lane (base lane + t), columns [col, col + 32).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

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
// B, the tile slices, K-major with the 64-byte swizzle: rows of 32 bf16
// (64 bytes), 8-row atoms of 512 bytes, the 16-byte chunk c of row r at chunk
// position c ^ ((r >> 1) & 3); SBO = 512 bytes between 8-row groups (LBO is
// not used by K-major swizzled layouts).
__device__ __forceinline__ uint64_t desc_b_sw64(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) | (1ull << 46) |
           (4ull << 61);
}
// byte offset of the 16-byte chunk (m >> 3) of lag row k in an A slice
__device__ __forceinline__ uint32_t a_chunk(int k, int mg) {
    return (uint32_t)((mg >> 3) * 4096 + (k >> 3) * 1024 + (k & 7) * 128 + (((mg & 7) ^ (k & 7)) << 4));
}
// byte offset of the 16-byte chunk kc (columns 8 kc .. 8 kc + 7) of tile row n in a B slice
__device__ __forceinline__ uint32_t b_chunk(int n, int kc) {
    return (uint32_t)((n >> 3) * 512 + (n & 7) * 64 + ((kc ^ ((n & 7) >> 1)) << 4));
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

// s + c += v with the rounding error of s + v kept in c (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float& s, float& c, float v) {
    const float t = s + v;
    const float bp = t - s;
    const float e = (s - (t - bp)) + (v - bp);
    s = t;
    c += e;
}

__device__ __forceinline__ void producer_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// Merged task of the tensor-core list: x, y = tiles of s1 and s2 (the zero
// tile if absent), z = cb | k << 16 | (part | variant << 2) << 26.
__device__ __forceinline__ int pk_cb(uint4 d) { return (int)(d.z & 0xFFFFu); }
__device__ __forceinline__ int pk_k(uint4 d) { return (int)((d.z >> 16) & 0x3FFu); }
__device__ __forceinline__ int pk_code(uint4 d) { return (int)(d.z >> 26); }

// Coefficient transform of a task: its variant for l and s, 3 for the
// windowed sums (used as stored).
__device__ __forceinline__ int task_xform(int code) { return (code & 3) == 2 ? 3 : (code >> 2) & 3; }

template <int NS>
struct TcLayout {
    static constexpr int NBARS = 2 * NS + 2 * NB + 1;  // + one barrier for the final MMA drain
    static constexpr size_t BARS = (size_t)NS * STAGE;
    static constexpr size_t SLOT = BARS + ((8 * NBARS + 15) / 16) * 16;  // TMEM address, abort flag
    static constexpr size_t DESC = SLOT + 16;                             // TC_CHUNK packed tasks (uint4)
    static constexpr size_t COLS = DESC + 16 * TC_CHUNK;                  // column order of the row block (uint16)
    static size_t bytes(int npad) { return COLS + (((size_t)npad * 2 + 15) / 16) * 16 + 1024; }
    static_assert(BARS % 1024 == 0 && SLOT % 16 == 0 && DESC % 16 == 0 && COLS % 16 == 0,
                  "shared-memory regions must keep their alignment (uint4 task loads)");
};

template <int NS>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_hist_tc(const uint4* __restrict__ tasks, const HistChunk* __restrict__ chunks,
              const __nv_bfloat16* __restrict__ tiles16,
              const __nv_bfloat16* __restrict__ ring16, const __nv_bfloat16* __restrict__ win16, long long step_i,
              int R, int npad, int C2, const int* __restrict__ colidx, double eta, double etap,
              double* __restrict__ partial, int* __restrict__ err) {
    using L = TcLayout<NS>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // swizzled operand atoms need 1 KB alignment: the launch adds 1 KB of slack
    unsigned char* smem = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sbase = su32(smem);
    const uint32_t bar0 = sbase + (uint32_t)L::BARS;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L::SLOT);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    uint4* sdesc = reinterpret_cast<uint4*>(smem + L::DESC);
    uint16_t* scol = reinterpret_cast<uint16_t*>(smem + L::COLS);
    // FULL: the coefficient rows (one arrival per copying thread, when its
    // cp.async copies have landed) and the tile slices (bytes of the bulk
    // copies, added to the barrier's transaction count) of a stage
    auto FULL = [&](int s) { return bar0 + 8u * s; };
    auto EMPTY = [&](int s) { return bar0 + 8u * (NS + s); };  // MMAs done with the stage
    auto ACCF = [&](int b) { return bar0 + 8u * (2 * NS + b); };
    auto ACCE = [&](int b) { return bar0 + 8u * (2 * NS + NB + b); };
    const uint32_t DRAIN = bar0 + 8u * (2 * NS + 2 * NB);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const HistChunk ch = chunks[blockIdx.x];
    const int ntask = ch.count;  // <= TC_CHUNK

    // the chunk's task list and the row block's column order, staged once
    for (int i = tid; i < ntask; i += TC_THREADS) sdesc[i] = tasks[ch.first + i];
    for (int p = tid; p < npad; p += TC_THREADS) scol[p] = (uint16_t)colidx[(size_t)ch.rb * npad + p];
    if (tid == 0) {
        for (int s = 0; s < NS; s++) {
            mbar_init(FULL(s), NPROD);
            mbar_init(EMPTY(s), 1);
        }
        for (int b = 0; b < NB; b++) {
            mbar_init(ACCF(b), 1);
            mbar_init(ACCE(b), NEPI / 32);
        }
        mbar_init(DRAIN, 1);
        *abort_flag = 0;
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

    if (warp < 2) {
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
        int issued = 0;  // tasks whose copies were issued
        bool ok = true;
        const size_t pstride = (size_t)npad * C2;  // elements of one bf16 slice of one panel
        // 16-byte pieces per coefficient row (C2 / 8); a batch below 64 waves
        // leaves the panel's upper columns uncopied (their TMEM lanes are never read)
        const int nch = C2 >> 3;
        for (int ti = 0; ti < ntask; ti++) {
            const uint4 d = sdesc[ti];
            const int cb = pk_cb(d), k = pk_k(d), code = pk_code(d);
            if (step_i - k < 1) continue;
            const int j = issued;
            const int s = j % NS;
            if (!mbar_wait(EMPTY(s), ((uint32_t)(j / NS) & 1u) ^ 1u, abort_flag, err, 2)) {
                ok = false;
                break;
            }
            if (t == 0) {  // slices in the order Y0 Z0 Y1 Z1 Y2 Z2; bytes added before this thread's arrival
                mbar_add_tx(FULL(s), STAGE_B);
#pragma unroll
                for (int q = 0; q < 3; q++) {
                    bulk_g2s(sbase + s * STAGE + STAGE_A + (2 * q) * B_SLICE, tiles16 + ((size_t)d.x * 3 + q) * (T * T),
                             B_SLICE, FULL(s));
                    bulk_g2s(sbase + s * STAGE + STAGE_A + (2 * q + 1) * B_SLICE,
                             tiles16 + ((size_t)d.y * 3 + q) * (T * T), B_SLICE, FULL(s));
                }
            }
            const int part = code & 3, var = (code >> 2) & 3;
            const __nv_bfloat16* pan = part == 2 ? win16 + (size_t)k * 3 * pstride
                                                 : ring16 + (((size_t)(slot_i - k + (slot_i < k ? R : 0)) * 2 + part) * 3) * pstride;
            const int swap = (part != 2 && var == 2) ? nch >> 1 : 0;  // [-v, u]: the u and v halves exchanged
            const uint32_t adst = sbase + s * STAGE;
#pragma unroll
            for (int ro = 0; ro < 4; ro++) {
                const __nv_bfloat16* row = pan + (size_t)scol[cb * T + ro * 8 + l8] * C2;
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int mg = (2 * warp + h) * 4 + l3;
                    if (mg >= nch) continue;
                    const int sc = mg + swap < nch ? mg + swap : mg + swap - nch;
                    const __nv_bfloat16* src = row + sc * 8;
#pragma unroll
                    for (int q = 0; q < 3; q++) cp_async16(adst + q * A_SLICE + dofs[ro][h], src + (size_t)q * pstride);
                }
            }
            // this thread's arrival on the stage fires when its copies have landed
            cp_async_arrive_noinc(FULL(s));
            issued = j + 1;
        }
        cp_async_wait_all();
        if (!ok && t == 0)  // let the tile copies in flight land before the CTA exits
            for (int jj = issued > NS ? issued - NS : 0; jj < issued; jj++)
                mbar_wait_drain(FULL(jj % NS), (uint32_t)(jj / NS) & 1u);
    } else if (warp == 2) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            int j = 0, g = -1, ing = 0, cur = -1;
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
                    if (!mbar_wait(ACCE(b), ((uint32_t)(g / NB) & 1u) ^ 1u, abort_flag, err, 3)) break;
                    tc_fence_after();
                    dcol = tmem + (uint32_t)(b * BUFCOLS);
                }
                const int s = j % NS;
                if (!mbar_wait(FULL(s), (uint32_t)(j / NS) & 1u, abort_flag, err, 4)) break;
                fence_proxy_async();  // coefficient rows written by cp.async (generic proxy)
                tc_fence_after();
                const uint32_t a0 = sbase + s * STAGE, b0 = a0 + STAGE_A;
                // K-half kk: A rows 16 kk .. 16 kk + 15 (two 1 KB row groups),
                // B columns 16 kk .. (32 bytes into each 64-byte row)
#pragma unroll
                for (int kk = 0; kk < 2; kk++) {
                    const uint64_t bd = desc_b_sw64(b0 + kk * 32);
                    mma_bf16(dcol, desc_a_sw128(a0 + kk * 2048), bd, idesc_bf16(192), (ing > 0 || kk > 0) ? 1u : 0u);
                    mma_bf16(dcol + 64, desc_a_sw128(a0 + A_SLICE + kk * 2048), bd, idesc_bf16(128), 1u);
                    mma_bf16(dcol + 128, desc_a_sw128(a0 + 2 * A_SLICE + kk * 2048), bd, idesc_bf16(64), 1u);
                }
                tc_commit(EMPTY(s));
                ing++;
                j++;
            }
            // the last (or interrupted) group: its commit also tells the
            // epilogue that every MMA issued by this thread has completed
            if (g >= 0) tc_commit(ACCF(g % NB));
            // TMEM is released only after every MMA of this CTA has completed
            tc_commit(DRAIN);
            mbar_wait_drain(DRAIN, 0);
        }
        __syncwarp();
    } else {
        // ---------------- epilogue ----------------
        const int quarter = warp & 3;  // TMEM lanes [32 quarter, 32 quarter + 32)
        const int m = quarter * 32 + lane;
        const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
        float hs0[32], hc0[32], hs1[32], hc1[32];  // compensated sums of s1 and s2
#pragma unroll
        for (int n = 0; n < 32; n++) hs0[n] = hc0[n] = hs1[n] = hc1[n] = 0.f;
        // per-column scale of each coefficient transform (u columns m < 64, v columns m >= 64)
        const bool ucol = m < C2 / 2;
        const float xs0 = ucol ? (float)eta : (float)(1.0 / eta), xs1 = ucol ? (float)etap : (float)(1.0 / etap),
                    xs2 = ucol ? -1.f : 1.f;
        // folds buffer b (transform key) into the sums of output o
        auto fold = [&](uint32_t col, float c, float (&hs)[32], float (&hc)[32], bool release, int b) {
            float va[32], vb[32];
            tmem_ld32(col + 64, va);   // terms of relative size 2^-8
            tmem_ld32(col + 128, vb);  // and 2^-16
            tmem_wait_ld();
#pragma unroll
            for (int n = 0; n < 32; n++) hc[n] += c * (va[n] + vb[n]);
            tmem_ld32(col, va);  // the leading products
            tmem_wait_ld();
            if (release) {
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(ACCE(b));
            }
#pragma unroll
            for (int n = 0; n < 32; n++) two_sum(hs[n], hc[n], c * va[n]);
        };
        auto drain = [&](int gg, int key) -> bool {
            const int b = gg % NB;
            if (!mbar_wait(ACCF(b), (uint32_t)(gg / NB) & 1u, abort_flag, err, 5)) return false;
            tc_fence_after();
            __syncwarp();
            const float c = key == 0 ? xs0 : key == 1 ? xs1 : key == 2 ? xs2 : 1.f;
            const uint32_t col = tl + (uint32_t)(b * BUFCOLS);
            fold(col, c, hs0, hc0, false, b);
            fold(col + 32, c, hs1, hc1, true, b);
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
        if (m < C2) {
            double* p0 = partial + (size_t)blockIdx.x * 2 * T * C2 + m;
            double* p1 = p0 + (size_t)T * C2;
#pragma unroll
            for (int n = 0; n < 32; n++) {
                p0[(size_t)n * C2] = (double)hs0[n] + (double)hc0[n];
                p1[(size_t)n * C2] = (double)hs1[n] + (double)hc1[n];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 2) {
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
}

// src: npanels panels of n doubles; dst: npanels x 3 bf16 slices of n values.
__global__ void k_split3(size_t n, int npanels, const double* __restrict__ src, __nv_bfloat16* __restrict__ dst) {
    const size_t total = n * (size_t)npanels;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t p = i / n, r = i - p * n;
        const double x = src[i];
        const __nv_bfloat16 a = __double2bfloat16(x);
        const double r1 = x - (double)__bfloat162float(a);
        const __nv_bfloat16 b = __double2bfloat16(r1);
        const double r2 = r1 - (double)__bfloat162float(b);
        const __nv_bfloat16 c = __double2bfloat16(r2);
        __nv_bfloat16* d = dst + p * 3 * n + r;
        d[0] = a;
        d[n] = b;
        d[2 * n] = c;
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
        unsigned char* d = reinterpret_cast<unsigned char*>(dst + (size_t)t * 3 * T * T) + b_chunk(r, kc);
        *reinterpret_cast<uint4*>(d) = make_uint4(pack2(a[0], a[1]), pack2(a[2], a[3]), pack2(a[4], a[5]), pack2(a[6], a[7]));
        *reinterpret_cast<uint4*>(d + B_SLICE) =
            make_uint4(pack2(b[0], b[1]), pack2(b[2], b[3]), pack2(b[4], b[5]), pack2(b[6], b[7]));
        *reinterpret_cast<uint4*>(d + 2 * B_SLICE) =
            make_uint4(pack2(c[0], c[1]), pack2(c[2], c[3]), pack2(c[4], c[5]), pack2(c[6], c[7]));
    }
}

// bf16 slices of l and s of one ring slot, columns [u | v], from the FP64
// ring's [-v, u] variant of each part: dst [2 parts][3 slices][npad][2B].
__global__ void k_split_ring(int npad, int B, const double* __restrict__ ring_slot, __nv_bfloat16* __restrict__ dst) {
    const int C2 = 2 * B;
    const size_t ps = (size_t)npad * C2;
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
        __nv_bfloat16* d = dst + (size_t)part * 3 * ps + r * C2 + m;
        d[0] = a;
        d[ps] = b;
        d[2 * ps] = __double2bfloat16(r2);
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
    const int blocks = (int)std::min<size_t>((2 * bv + 255) / 256, 152 * 16);
    k_split_ring<<<blocks, 256, 0, s>>>(h->npad, h->B, h->d_ring + (size_t)slot * 6 * bv,
                                        reinterpret_cast<__nv_bfloat16*>(h->d_ring16) + (size_t)slot * 6 * bv);
    h->launches++;
}


// pipeline depth: the deepest that fits next to the row block's column order
int history_tc_stages(int npad) {
    if (npad > 65536) return 0;
    if (TcLayout<6>::bytes(npad) <= TC_SMEM_MAX) return 6;
    if (TcLayout<5>::bytes(npad) <= TC_SMEM_MAX) return 5;
    if (TcLayout<4>::bytes(npad) <= TC_SMEM_MAX) return 4;
    return 0;
}

bool history_tc_fits(int npad) { return history_tc_stages(npad) > 0; }

void launch_split3(mot_handle* h, int npanels, const double* src, uint16_t* dst, cudaStream_t s) {
    const size_t n = (size_t)h->npad * 2 * h->B;
    const size_t total = n * (size_t)npanels;
    if (total == 0) return;
    const int blocks = (int)std::min<size_t>((total + 255) / 256, 152 * 16);
    k_split3<<<blocks, 256, 0, s>>>(n, npanels, src, reinterpret_cast<__nv_bfloat16*>(dst));
    h->launches++;
}

void launch_history_tc(mot_handle* h, const TaskList& tl, long long step_i, double* out_s1, double* out_s2,
                       cudaStream_t s) {
    const int C2 = 2 * h->B;
    if (tl.nchunks > 0) {
        const bool timed = h->opt.timing && h->ev0 && step_i > h->K;
        if (timed) cudaEventRecord(h->ev0, s);
        static std::atomic<unsigned long long> attr{0};
        once_per_device(attr, h->dev, [] {
            cudaFuncSetAttribute(k_hist_tc<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM_MAX);
            cudaFuncSetAttribute(k_hist_tc<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM_MAX);
            cudaFuncSetAttribute(k_hist_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM_MAX);
        });
        const uint4* pt = tl.packed;
        const auto* r16 = reinterpret_cast<const __nv_bfloat16*>(h->d_ring16);
        const auto* w16 = reinterpret_cast<const __nv_bfloat16*>(h->d_win16);
        switch (history_tc_stages(h->npad)) {
            case 6:
                k_hist_tc<6><<<tl.nchunks, TC_THREADS, TcLayout<6>::bytes(h->npad), s>>>(
                    pt, tl.chunks, reinterpret_cast<const __nv_bfloat16*>(h->d_tiles16), r16, w16, step_i, h->R, h->npad, C2, h->d_colidx, h->eta, h->etap,
                    h->d_partial, h->d_cg_iters + 2);
                break;
            case 5:
                k_hist_tc<5><<<tl.nchunks, TC_THREADS, TcLayout<5>::bytes(h->npad), s>>>(
                    pt, tl.chunks, reinterpret_cast<const __nv_bfloat16*>(h->d_tiles16), r16, w16, step_i, h->R, h->npad, C2, h->d_colidx, h->eta, h->etap,
                    h->d_partial, h->d_cg_iters + 2);
                break;
            default:
                k_hist_tc<4><<<tl.nchunks, TC_THREADS, TcLayout<4>::bytes(h->npad), s>>>(
                    pt, tl.chunks, reinterpret_cast<const __nv_bfloat16*>(h->d_tiles16), r16, w16, step_i, h->R, h->npad, C2, h->d_colidx, h->eta, h->etap,
                    h->d_partial, h->d_cg_iters + 2);
        }
        if (timed) {
            cudaEventRecord(h->ev1, s);
            h->ev_pending = true;
        }
        h->launches++;
    }
    k_hist_reduce_idx<<<h->nrb, 256, 0, s>>>(tl.rb_ptr, tl.rb_chunks, h->d_partial, C2, out_s1, out_s2);
    h->launches++;
}

}  // namespace mot
