// FP64-accurate dense products on the tensor cores by exact integer slices
// (sm_100 family): Y = A X with A a fixed M x K FP64 matrix of the mixed path
// (the left factor [M1 | M2], Q_0) and X a K x N FP64 block vector.
//
// Method: the error-free splitting of Ozaki et al. (the "Ozaki scheme": each
// operand written as a sum of slices whose pairwise products are exact in the
// low-precision unit, the slice products summed in higher precision), here in
// its integer form -- fixed-point slices of a common per-row / per-column
// power-of-two scale, so that the tensor core's FP32 accumulation of a chunk
// is itself exact.
//
// Every row of A is scaled by a power of two so that |A_ik| < 1, every column
// of X likewise; each scaled value is split into S signed 7-bit integer
// slices, a = sum_p a_p 2^(-6 - 7(p-1)), |a_p| <= 64, held exactly in bf16.
// The product of two slices is an integer of magnitude <= 2^12, exact in the
// tensor core's FP32 accumulator; slice pairs are accumulated by weight
// level L = p + q - 2 (pairs with p + q <= S + 1: S levels), over K chunks of
// 128, so that every partial sum stays an integer below 2^22 and the FP32
// accumulation is exact. After each chunk the epilogue folds the S levels,
// scaled by 2^(-7L) (exact), into a compensated FP32 pair per output element;
// the result is scaled back in FP64. The dropped levels and the slice
// representation leave a relative error of about 2^(-7S + 2) of
// sum_k |A_ik| |X_kj|: S = 6 (21 pairs) for FP64-accurate products, S = 4
// (10 pairs, ~2^-26) for the products the FP32 solves need.
//
// Slices are stacked along N so that one MMA covers a whole row of the
// product table: A_p x [X_1; ...; X_(S+1-p)] (N = 64 (S + 1 - p)) into TMEM
// columns [64 (p-1), 64 S), i.e. level p + q - 2 of every q. Operands are pre-arranged
// in the K-major 64-byte-swizzled layout (rows of 32 bf16), A once at set-up
// and X per call, so one bulk copy per operand moves a pipeline stage.
//
// Warp roles (192 threads, one CTA per SM): warp 0 copies, warp 1 allocates
// TMEM and issues the MMAs (lane 0), warps 2-5 fold TMEM into the sums (one
// output row per thread, 64 columns). Every mbarrier wait is bounded in time
// and ends in an error status.
#include <cuda_bf16.h>

#include <algorithm>

#include "mot_internal.h"
#include "tc_ptx.h"

namespace {

using namespace tcx;

constexpr int EM = 128;           // rows of A per CTA
constexpr int EN = 64;            // columns of X per CTA
constexpr int EK = 32;            // K per pipeline stage (one 64-byte row of bf16)
constexpr int KC_TILES = 4;       // stages per exact accumulation chunk (K = 128)
constexpr int A_TILE = EM * EK * 2;          // 8192 bytes per slice
constexpr int B_TILE = EN * EK * 2;          // 4096 bytes per slice
constexpr int E_THREADS = 192;
constexpr int E_TMEM = 512;                  // >= 64 S

// layout of the S-slice variant
template <int S>
struct EmuCfg {
    static constexpr int A_STAGE = S * A_TILE;
    static constexpr int B_STAGE = S * B_TILE;
    static constexpr int STAGE = A_STAGE + B_STAGE;
    static constexpr int NS = (int)((227 * 1024 - 2048) / STAGE);  // pipeline stages
    static constexpr int NBARS = 2 * NS + 3;                        // FULL, EMPTY, ACCF, ACCE, DRAIN
    static constexpr size_t SMEM = (size_t)NS * STAGE + 8 * NBARS + 16 + 1024;
    static_assert(S * EN <= E_TMEM, "TMEM");
    static_assert(STAGE % 1024 == 0, "stage alignment");
    static_assert(SMEM <= 227 * 1024 && NS >= 2, "shared memory");
};

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// S signed 7-bit slices of a (|a| < 1): a = sum_p s[p] 2^(-6 - 7p)
template <int S>
__device__ __forceinline__ void slice_n(double a, float (&s)[S]) {
    double t = a * 64.0;
#pragma unroll
    for (int p = 0; p < S; p++) {
        const double r = rint(t);
        s[p] = (float)r;
        t = (t - r) * 128.0;
    }
}

__device__ __forceinline__ void twosum(float& s, float& c, float v) {
    const float t = s + v;
    const float bp = t - s;
    const float e = (s - (t - bp)) + (v - bp);
    s = t;
    c += e;
}

// exponent e with |x| / 2^e < 1 for all x of the row (0 for a zero row)
__global__ void k_row_exponents(int M, int Mp, int K, const double* __restrict__ A, int* __restrict__ ea) {
    const int i = blockIdx.x;
    double m = 0.0;
    if (i < M)
        for (int k = threadIdx.x; k < K; k += blockDim.x) m = fmax(m, fabs(A[(size_t)i * K + k]));
    __shared__ double red[256];
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int e = 0;
        if (red[0] > 0.0) frexp(red[0], &e);
        ea[i] = e;
    }
}

// A (M x K, row-major) -> slices in [Mp / 128][K / 32][S][128 x 32, 64-byte swizzle]
template <int NSL>
__global__ void k_slice_rows(int M, int Mp, int K, const double* __restrict__ A, const int* __restrict__ ea,
                             __nv_bfloat16* __restrict__ A16) {
    const int KT = K / EK;
    const long long total = (long long)Mp * (K / 8);
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / (K / 8)), k8 = (int)(idx - (long long)i * (K / 8));
        float s[8][NSL];
#pragma unroll
        for (int e = 0; e < 8; e++) {
            const double a = i < M ? ldexp(A[(size_t)i * K + k8 * 8 + e], -ea[i]) : 0.0;
            slice_n<NSL>(a, s[e]);
        }
        const int mt = i / EM, r = i % EM, kt = (k8 * 8) / EK, kc = ((k8 * 8) % EK) / 8;
        unsigned char* base = reinterpret_cast<unsigned char*>(A16 + (((size_t)mt * KT + kt) * NSL) * (EM * EK));
#pragma unroll
        for (int p = 0; p < NSL; p++) {
            __nv_bfloat16 b[8];
#pragma unroll
            for (int e = 0; e < 8; e++) b[e] = __float2bfloat16_rn(s[e][p]);  // integers |v| <= 64: exact
            *reinterpret_cast<uint4*>(base + (size_t)p * A_TILE + sw64_chunk(r, kc)) =
                make_uint4(pack2(b[0], b[1]), pack2(b[2], b[3]), pack2(b[4], b[5]), pack2(b[6], b[7]));
        }
    }
}

// exponent of every column of X (K x N, row-major)
__global__ void k_col_exponents(int K, int N, const double* __restrict__ X, int* __restrict__ ex) {
    const int j = blockIdx.x;
    double m = 0.0;
    for (int k = threadIdx.x; k < K; k += blockDim.x) m = fmax(m, fabs(X[(size_t)k * N + j]));
    __shared__ double red[256];
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int e = 0;
        if (red[0] > 0.0) frexp(red[0], &e);
        ex[j] = e;
    }
}

// X (K x N) -> slices of X^T in [NH][K / 32][S][64 x 32, 64-byte swizzle]
template <int NSL>
__global__ void k_slice_cols(int K, int N, int NH, const double* __restrict__ X, const int* __restrict__ ex,
                             __nv_bfloat16* __restrict__ X16) {
    const int KT = K / EK;
    const long long total = (long long)NH * EN * (K / 8);
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int n = (int)(idx % (NH * EN)), k8 = (int)(idx / (NH * EN));
        float s[8][NSL];
#pragma unroll
        for (int e = 0; e < 8; e++) {
            const double x = n < N ? ldexp(X[(size_t)(k8 * 8 + e) * N + n], -ex[n]) : 0.0;
            slice_n<NSL>(x, s[e]);
        }
        const int nh = n / EN, r = n % EN, kt = (k8 * 8) / EK, kc = ((k8 * 8) % EK) / 8;
        unsigned char* base = reinterpret_cast<unsigned char*>(X16 + (((size_t)nh * KT + kt) * NSL) * (EN * EK));
#pragma unroll
        for (int q = 0; q < NSL; q++) {
            __nv_bfloat16 b[8];
#pragma unroll
            for (int e = 0; e < 8; e++) b[e] = __float2bfloat16_rn(s[e][q]);
            *reinterpret_cast<uint4*>(base + (size_t)q * B_TILE + sw64_chunk(r, kc)) =
                make_uint4(pack2(b[0], b[1]), pack2(b[2], b[3]), pack2(b[4], b[5]), pack2(b[6], b[7]));
        }
    }
}

// Y[z] (M x N, rows < M, columns < N) = partial product over the k-tiles
// [z * kts, (z + 1) * kts) of CTA split z (gridDim.z splits; kts a multiple
// of KC_TILES).
template <int NSL>
__global__ void __launch_bounds__(E_THREADS, 1)
    k_emu_gemm(int M, int N, int K, int kts, const __nv_bfloat16* __restrict__ A16, const int* __restrict__ ea,
               const __nv_bfloat16* __restrict__ X16, const int* __restrict__ ex, double* __restrict__ Y,
               int* __restrict__ err) {
    using C = EmuCfg<NSL>;
    constexpr int E_NS = C::NS, E_STAGE = C::STAGE, A_STAGE = C::A_STAGE, B_STAGE = C::B_STAGE;
    constexpr int NLEV = NSL;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sbase = su32(smem);
    const uint32_t bar0 = sbase + E_NS * E_STAGE;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + E_NS * E_STAGE + 8 * C::NBARS);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    auto FULL = [&](int s) { return bar0 + 8u * s; };
    auto EMPTY = [&](int s) { return bar0 + 8u * (E_NS + s); };
    const uint32_t ACCF = bar0 + 8u * (2 * E_NS), ACCE = ACCF + 8u, DRAIN = ACCF + 16u;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mt = blockIdx.x, nh = blockIdx.y, z = blockIdx.z;
    const int KT = K / EK;
    const int kt0 = z * kts, kt1 = min(KT, kt0 + kts);
    const int ntile = max(0, kt1 - kt0);
    const int nchunk = (ntile + KC_TILES - 1) / KC_TILES;

    if (tid == 0) {
        for (int s = 0; s < E_NS; s++) {
            mbar_init(FULL(s), 1);
            mbar_init(EMPTY(s), 1);
        }
        mbar_init(ACCF, 1);
        mbar_init(ACCE, 4);
        mbar_init(DRAIN, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 1) {
        tmem_alloc(su32(tmem_slot), E_TMEM);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------- copies ----------------
        if (lane == 0) {
            int issued = 0;
            for (int j = 0; j < ntile; j++) {
                const int s = j % E_NS;
                if (!mbar_wait(EMPTY(s), ((uint32_t)(j / E_NS) & 1u) ^ 1u, abort_flag, err, 11)) break;
                const int kt = kt0 + j;
                mbar_expect_tx(FULL(s), E_STAGE);
                bulk_g2s(sbase + s * E_STAGE, A16 + (((size_t)mt * KT + kt) * NSL) * (EM * EK), A_STAGE, FULL(s));
                bulk_g2s(sbase + s * E_STAGE + A_STAGE, X16 + (((size_t)nh * KT + kt) * NSL) * (EN * EK), B_STAGE,
                         FULL(s));
                issued = j + 1;
            }
            if (*abort_flag)  // let the copies in flight land before the CTA exits
                for (int jj = issued > E_NS ? issued - E_NS : 0; jj < issued; jj++)
                    mbar_wait_drain(FULL(jj % E_NS), (uint32_t)(jj / E_NS) & 1u);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- MMA issue ----------------
        if (lane == 0) {
            for (int j = 0; j < ntile; j++) {
                const int c = j / KC_TILES, first = (j % KC_TILES) == 0;
                if (first) {
                    if (!mbar_wait(ACCE, ((uint32_t)c & 1u) ^ 1u, abort_flag, err, 12)) break;
                    tc_fence_after();
                }
                const int s = j % E_NS;
                if (!mbar_wait(FULL(s), (uint32_t)(j / E_NS) & 1u, abort_flag, err, 13)) break;
                tc_fence_after();
                const uint32_t a0 = sbase + s * E_STAGE, b0 = a0 + A_STAGE;
#pragma unroll
                for (int kk = 0; kk < 2; kk++) {
#pragma unroll
                    for (int p = 1; p <= NSL; p++) {
                        const int rows = EN * (NSL + 1 - p);  // X slices 1 .. S + 1 - p stacked
                        const uint64_t ad = desc_kmajor_sw64(a0 + (p - 1) * A_TILE + kk * 32);
                        const uint32_t acc = (first && kk == 0 && p == 1) ? 0u : 1u;
                        const int n0 = rows > 256 ? 256 : rows;
                        mma_bf16(tmem + (uint32_t)(EN * (p - 1)), ad, desc_kmajor_sw64(b0 + kk * 32),
                                 idesc_bf16_kk(n0), acc);
                        if (rows > 256)
                            mma_bf16(tmem + (uint32_t)(EN * (p - 1) + 256), ad,
                                     desc_kmajor_sw64(b0 + 256 * 64 + kk * 32), idesc_bf16_kk(rows - 256), acc);
                    }
                }
                tc_commit(EMPTY(s));
                if ((j % KC_TILES) == KC_TILES - 1 || j == ntile - 1) tc_commit(ACCF);
            }
            tc_commit(DRAIN);
            mbar_wait_drain(DRAIN, 0);
        }
        __syncwarp();
    } else {
        // ---------------- fold: one output row per thread ----------------
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
        float hi[EN], lo[EN];
#pragma unroll
        for (int n = 0; n < EN; n++) hi[n] = lo[n] = 0.f;
        bool ok = true;
        for (int c = 0; c < nchunk && ok; c++) {
            if (!mbar_wait(ACCF, (uint32_t)c & 1u, abort_flag, err, 14)) {
                ok = false;
                break;
            }
            tc_fence_after();
            __syncwarp();
#pragma unroll
            for (int L = NLEV - 1; L >= 0; L--) {  // small levels first
                const float w = ldexpf(1.f, -7 * L);
#pragma unroll
                for (int hh = 0; hh < 2; hh++) {
                    float v[32];
                    tmem_ld32(tl + (uint32_t)(EN * L + 32 * hh), v);
                    tmem_wait_ld();
#pragma unroll
                    for (int n = 0; n < 32; n++) twosum(hi[32 * hh + n], lo[32 * hh + n], v[n] * w);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(ACCE);
        }
        const int gi = mt * EM + row;
        if (ok && gi < M) {
            double* out = Y + (size_t)z * M * N + (size_t)gi * N;
#pragma unroll
            for (int n = 0; n < EN; n++) {
                const int gj = nh * EN + n;
                if (gj < N) out[gj] = ldexp((double)hi[n] + (double)lo[n], ea[gi] + ex[gj] - 12);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, E_TMEM);
    }
}

__global__ void k_emu_reduce(size_t n, int S, const double* __restrict__ W, double* __restrict__ Y) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int z = 0; z < S; z++) v += W[(size_t)z * n + i];
        Y[i] = v;
    }
}

}  // namespace

namespace mot {

int emu_prepare(mot_handle* h, const double* A, int M, int K, EmuMat* out, int nsl) {
    if (K % EK != 0) return fail(h, MOT_EINVAL, "emulated FP64 product: K must be a multiple of 32");
    if (nsl != 4 && nsl != 6) return fail(h, MOT_EINVAL, "emulated product: 4 or 6 slices");
    out->nsl = nsl;
    out->M = M;
    out->K = K;
    out->Mp = (M + EM - 1) / EM * EM;
    out->ea = (int*)dalloc(h, sizeof(int) * out->Mp);
    out->a16 = (uint16_t*)dalloc(h, sizeof(uint16_t) * (size_t)nsl * out->Mp * K);
    if (!out->ea || !out->a16) return fail(h, MOT_EOOM, "device allocation (emulated FP64 operator)");
    k_row_exponents<<<out->Mp, 256>>>(M, out->Mp, K, A, out->ea);
    const long long total = (long long)out->Mp * (K / 8);
    const int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 64);
    if (nsl == 6)
        k_slice_rows<6><<<blocks, 256>>>(M, out->Mp, K, A, out->ea, reinterpret_cast<__nv_bfloat16*>(out->a16));
    else
        k_slice_rows<4><<<blocks, 256>>>(M, out->Mp, K, A, out->ea, reinterpret_cast<__nv_bfloat16*>(out->a16));
    h->launches += 2;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "emulated FP64 operator set-up");
    return MOT_OK;
}

void emu_free(mot_handle* h, EmuMat* m) {
    if (m->ea) cudaFree(m->ea);
    if (m->a16) cudaFree(m->a16);
    m->ea = nullptr;
    m->a16 = nullptr;
}

int launch_emu_gemm(mot_handle* h, const EmuMat& A, const double* X, int N, double* Y, cudaStream_t s) {
    const int K = A.K, KT = K / EK, NH = (N + EN - 1) / EN, MT = A.Mp / EM;
    int nsm = 148;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->dev);
    // K splits so that the grid covers the SMs; each split a multiple of a chunk
    int S = std::max(1, std::min(nsm / std::max(1, MT * NH), (KT + KC_TILES - 1) / KC_TILES));
    int kts = ((KT + S - 1) / S + KC_TILES - 1) / KC_TILES * KC_TILES;
    S = (KT + kts - 1) / kts;
    const int NSL = A.nsl;
    const size_t x16 = sizeof(uint16_t) * (size_t)NH * KT * NSL * EN * EK;
    const size_t part = S > 1 ? sizeof(double) * (size_t)S * A.M * N : 0;
    const size_t need = x16 + part + sizeof(int) * 256;
    if (need > h->emuws_bytes) {
        if (h->d_emuws) {
            cudaFree(h->d_emuws);
            h->device_bytes -= (int64_t)h->emuws_bytes;
        }
        h->emuws_bytes = 0;
        h->d_emuws = (unsigned char*)dalloc(h, need);
        if (!h->d_emuws) return fail(h, MOT_EOOM, "device allocation (emulated FP64 workspace)");
        h->emuws_bytes = need;
    }
    if (N > 256) return fail(h, MOT_EINVAL, "emulated FP64 product: N > 256");
    double* ws = reinterpret_cast<double*>(h->d_emuws);
    __nv_bfloat16* d_x16 = reinterpret_cast<__nv_bfloat16*>(h->d_emuws + part);
    int* d_ex = reinterpret_cast<int*>(h->d_emuws + part + x16);
    k_col_exponents<<<N, 256, 0, s>>>(K, N, X, d_ex);
    const long long total = (long long)NH * EN * (K / 8);
    const int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 32);
    static std::atomic<unsigned long long> attr{0};
    once_per_device(attr, h->dev, [] {
        cudaFuncSetAttribute(k_emu_gemm<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EmuCfg<6>::SMEM);
        cudaFuncSetAttribute(k_emu_gemm<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EmuCfg<4>::SMEM);
    });
    dim3 grid(MT, NH, S);
    const auto* a16 = reinterpret_cast<const __nv_bfloat16*>(A.a16);
    double* out = S > 1 ? ws : Y;
    if (NSL == 6) {
        k_slice_cols<6><<<blocks, 256, 0, s>>>(K, N, NH, X, d_ex, d_x16);
        k_emu_gemm<6><<<grid, E_THREADS, EmuCfg<6>::SMEM, s>>>(A.M, N, K, kts, a16, A.ea, d_x16, d_ex, out,
                                                               h->d_cg_iters + 2);
    } else {
        k_slice_cols<4><<<blocks, 256, 0, s>>>(K, N, NH, X, d_ex, d_x16);
        k_emu_gemm<4><<<grid, E_THREADS, EmuCfg<4>::SMEM, s>>>(A.M, N, K, kts, a16, A.ea, d_x16, d_ex, out,
                                                               h->d_cg_iters + 2);
    }
    h->launches += 3;
    if (S > 1) {
        const size_t n = (size_t)A.M * N;
        k_emu_reduce<<<(int)std::min<size_t>((n + 255) / 256, 4096), 256, 0, s>>>(n, S, ws, Y);
        h->launches++;
    }
    return MOT_OK;
}

}  // namespace mot
