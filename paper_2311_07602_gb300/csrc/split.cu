// Split-precision path: C += A B with the operands cut into BF16/FP16 digit
// slices, the slice products on the 5th-generation tensor cores (tcgen05,
// FP32 accumulators in TMEM) and the recombination and the accumulation
// across k-chunks in binary64.
//
// The paper computes in binary64 only (Sec. 7); this path follows the
// error-free splitting of Ozaki, Ogita, Oishi and Rump (Numer. Algorithms
// 2012) with these choices, which define the result exactly:
//   * per k-chunk of kc columns, row i of A gets E_i with 2^(E_i-1) <=
//     max|a_ip| < 2^E_i and column j of B gets F_j likewise (0 for a zero
//     row/column);
//   * Z = RN_even(a 2^(beta S - E)) (one rounding of the exact value), then
//     balanced digits, lowest first: d_s = ((Z + 2^(beta-1)) mod 2^beta) -
//     2^(beta-1), Z = (Z - d_s) / 2^beta for s = S..2, d_1 = Z;
//   * pairs (s, t) with s + t <= S + 1 are multiplied; pairs of one level
//     L = s + t accumulate in one FP32 TMEM accumulator, exact because kc
//     keeps every level sum within 2^24 (BF16: beta 8, kc 128; FP16: beta 9,
//     kc 32);
//   * per chunk the level sums are combined exactly as a 64-bit integer
//     I = sum_L P_L 2^(beta (S+1-L)) (|I| < 2^53), turned into the binary64
//     value I 2^(E_i + F_j - beta (S+1)) without rounding, and added to a
//     binary64 accumulator that starts from C.
//
// Kernel shape: one CTA per 128 x 64 output tile, 128 threads, thread t owns
// row t of the tile (= TMEM lane t).  Per chunk the threads compute the
// exponents straight from global memory, then write the digit planes of A
// (128 x ks) and B (64 x ks) into shared memory in the K-major, no-swizzle
// core-matrix layout (8 rows x 16 bytes per core matrix; LBO 128 bytes
// between core matrices along k, SBO = ks/8 * 128 bytes between 8-row
// groups); one thread issues tcgen05.mma (M 128, N 64, K 16) for every kept
// pair and k16 step and commits to an mbarrier.  Waits on that mbarrier are
// bounded: on expiry the kernel records an error in the plan's status word,
// releases its TMEM and returns.
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "lrb_internal.h"
#include "split.h"

namespace lrb {
namespace split {

namespace {

constexpr int kTM = 128;       // tile rows (MMA M)
constexpr int kTN = 64;        // tile cols (MMA N)
constexpr int kThreadsS = 128;
constexpr int kTmemCols = 256; // S levels x 64 columns, rounded to a power of two
constexpr long long kSpinLimit = 1ll << 26;

struct SItem {
    int32_t entry, row0, col0, pad;
};

template <bool FP16, int S>
struct Cfg {
    static constexpr int beta = FP16 ? 9 : 8;
    static constexpr int kc = FP16 ? 32 : 128;     // exponent chunk
    static constexpr int ks = FP16 ? 32 : 64;      // staged sub-chunk
    static constexpr int planeA = kTM * ks * 2;    // bytes per digit plane of A
    static constexpr int planeB = kTN * ks * 2;
    static constexpr int sbo = ks / 8 * 128;
    static constexpr int smem = S * (planeA + planeB);
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t make_desc(uint32_t addr, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);          // start address
    d |= (uint64_t)(128 >> 4) << 16;                  // LBO: next core matrix along k
    d |= (uint64_t)(sbo >> 4) << 32;                  // SBO: next 8-row group
    d |= (uint64_t)1 << 46;                           // descriptor version (tcgen05)
    return d;                                         // base offset 0, no swizzle
}

template <bool FP16>
__device__ __forceinline__ uint32_t make_idesc() {
    uint32_t d = 0;
    d |= 1u << 4;                                      // D: F32
    d |= (FP16 ? 0u : 1u) << 7;                        // A: F16 / BF16
    d |= (FP16 ? 0u : 1u) << 10;                       // B: F16 / BF16
    d |= (uint32_t)(kTN >> 3) << 17;                   // N
    d |= (uint32_t)(kTM >> 4) << 24;                   // M
    return d;                                          // A, B K-major; dense
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long long i = 0; i < kSpinLimit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// |a| bit pattern (sign cleared) -> E with 2^(E-1) <= |a| < 2^E (a != 0).
__device__ __forceinline__ int exp_of_bits(unsigned long long mag) {
    const int ef = (int)(mag >> 52);
    if (ef) return ef - 1022;
    return (64 - __clzll((long long)mag)) - 1074;   // subnormal
}

// Balanced digits of a given the chunk exponent E (see file comment).
template <int S, int BETA>
__device__ __forceinline__ void make_digits(double a, int E, int (&d)[S]) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(a);
    const unsigned long long mag = bits & 0x7FFFFFFFFFFFFFFFull;
    long long Z = 0;
    if (mag != 0) {
        const int ef = (int)(mag >> 52);
        const unsigned long long M = (mag & 0xFFFFFFFFFFFFFull) | (ef ? (1ull << 52) : 0ull);
        const int e = (ef ? ef : 1) - 1075;                 // a = M 2^e
        const int sh = E - BETA * S - e;                     // Z = RN(M 2^-sh)
        if (sh <= 0) {
            Z = (long long)(M << (-sh));
        } else if (sh < 64) {
            const unsigned long long half = 1ull << (sh - 1);
            Z = (long long)((M + half - 1 + ((M >> sh) & 1ull)) >> sh);
        }
        if (bits >> 63) Z = -Z;
    }
    constexpr long long base = 1ll << BETA, h = 1ll << (BETA - 1);
#pragma unroll
    for (int s = S - 1; s >= 1; --s) {
        const long long dig = ((Z + h) & (base - 1)) - h;
        d[s] = (int)dig;
        Z = (Z - dig) >> BETA;
    }
    d[0] = (int)Z;
}

template <bool FP16>
__device__ __forceinline__ uint16_t digit_bits(int d) {
    const float f = (float)d;   // |d| <= 2^(beta): exact in float and in the 16-bit type
    if constexpr (FP16) {
        return __half_as_ushort(__float2half_rn(f));
    } else {
        return (uint16_t)(__float_as_uint(f) >> 16);
    }
}

// Exact binary64 of I 2^X for |I| < 2^53, built from the bits.
__device__ __forceinline__ double scaled_int_to_double(long long I, int X) {
    if (I == 0) return 0.0;
    const unsigned long long u = (unsigned long long)(I < 0 ? -I : I);
    const int lz = __clzll((long long)u);
    const int biased = 1023 + (63 - lz) + X;
    if (biased <= 0 || biased >= 2047) return ldexp((double)I, X);   // out of the normal range
    const unsigned long long mant = (u << (lz - 11)) & 0xFFFFFFFFFFFFFull;
    const unsigned long long b = (I < 0 ? (1ull << 63) : 0ull) | ((unsigned long long)biased << 52) | mant;
    return __longlong_as_double((long long)b);
}

template <bool FP16, int S>
__global__ void __launch_bounds__(kThreadsS, 2) k_split(const DevDesc* __restrict__ descs,
                                                         const SItem* __restrict__ items,
                                                         int* __restrict__ status,
                                                         float* __restrict__ dump) {
    using C_ = Cfg<FP16, S>;
    constexpr int BETA = C_::beta, KC = C_::kc, KS = C_::ks;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* planeA = smem;                                  // S planes of 128 x ks
    uint8_t* planeB = smem + S * C_::planeA;                 // S planes of 64 x ks
    __shared__ int s_F[kTN];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_tmem;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const SItem item = items[blockIdx.x];
    const DevDesc d = descs[item.entry];
    const int m0 = item.row0, n0 = item.col0;
    const int row = m0 + tid;
    const bool row_ok = row < d.m;
    const int wc = min(kTN, d.n - n0);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&s_bar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = s_tmem;
    const uint32_t bar = smem_u32(&s_bar);
    uint32_t phase = 0;
    bool failed = false;

    // binary64 accumulators: row `row`, columns n0 .. n0+63, starting from C
    double acc[kTN];
#pragma unroll
    for (int j = 0; j < kTN; ++j) acc[j] = 0.0;
    if (row_ok) {
#pragma unroll
        for (int j = 0; j < kTN; ++j)
            if (j < wc) acc[j] = d.C[(size_t)row + (size_t)(n0 + j) * (size_t)d.ldc];
    }

    const uint32_t idesc = make_idesc<FP16>();
    const int nchunks = (d.k + KC - 1) / KC;
    for (int c = 0; c < nchunks; ++c) {
        const int k0 = c * KC;
        const int kcl = min(KC, d.k - k0);
        // ---- exponents: row of A (this thread), columns of B (warp-wide) ----
        int E = 0;
        if (row_ok) {
            unsigned long long mx = 0;
            const double* a = d.A + (size_t)row + (size_t)k0 * (size_t)d.lda;
#pragma unroll 8
            for (int p = 0; p < kcl; ++p) {
                const unsigned long long v =
                    (unsigned long long)__double_as_longlong(__ldg(a + (size_t)p * (size_t)d.lda)) & 0x7FFFFFFFFFFFFFFFull;
                mx = v > mx ? v : mx;
            }
            E = mx ? exp_of_bits(mx) : 0;
        }
        for (int j = warp; j < kTN; j += kThreadsS / 32) {
            unsigned long long mx = 0;
            if (j < wc) {
                const double* b = d.B + (size_t)k0 + (size_t)(n0 + j) * (size_t)d.ldb;
                for (int p = lane; p < kcl; p += 32) {
                    const unsigned long long v =
                        (unsigned long long)__double_as_longlong(__ldg(b + p)) & 0x7FFFFFFFFFFFFFFFull;
                    mx = v > mx ? v : mx;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long w = __shfl_xor_sync(0xffffffffu, mx, o);
                mx = w > mx ? w : mx;
            }
            if (lane == 0) s_F[j] = mx ? exp_of_bits(mx) : 0;
        }
        __syncthreads();

        // ---- sub-chunks: digits to shared memory, then the tensor-core pass ----
        for (int h0 = 0; h0 < KC; h0 += KS) {
            const int kb = k0 + h0;                // first k of this sub-chunk
            if (kb >= d.k) break;                  // ragged last chunk
            const int kl = max(0, min(KS, d.k - kb));
            // A digits: this thread's row, KS columns, 8 at a time (16-byte stores)
            {
                const double* a = d.A + (size_t)row + (size_t)kb * (size_t)d.lda;
                uint8_t* dst = planeA + (tid >> 3) * C_::sbo + (tid & 7) * 16;
#pragma unroll 1
                for (int g = 0; g < KS / 8; ++g) {
                    uint32_t packed[S][4];
#pragma unroll
                    for (int q = 0; q < 8; q += 2) {
                        int dg0[S], dg1[S];
                        const int kk = g * 8 + q;
                        const double a0 = (row_ok && kk < kl) ? __ldg(a + (size_t)kk * (size_t)d.lda) : 0.0;
                        const double a1 = (row_ok && kk + 1 < kl) ? __ldg(a + (size_t)(kk + 1) * (size_t)d.lda) : 0.0;
                        make_digits<S, BETA>(a0, E, dg0);
                        make_digits<S, BETA>(a1, E, dg1);
#pragma unroll
                        for (int s = 0; s < S; ++s)
                            packed[s][q >> 1] = (uint32_t)digit_bits<FP16>(dg0[s]) |
                                                ((uint32_t)digit_bits<FP16>(dg1[s]) << 16);
                    }
#pragma unroll
                    for (int s = 0; s < S; ++s)
                        *reinterpret_cast<uint4*>(dst + s * C_::planeA + g * 128) =
                            make_uint4(packed[s][0], packed[s][1], packed[s][2], packed[s][3]);
                }
            }
            // B digits: warp w takes columns w, w+4, ...; lanes run along k
            for (int j = warp; j < kTN; j += kThreadsS / 32) {
                const int F = s_F[j];
                const double* b = d.B + (size_t)kb + (size_t)(n0 + j) * (size_t)d.ldb;
                uint8_t* dst = planeB + (j >> 3) * C_::sbo + (j & 7) * 16;
                for (int kk = lane; kk < KS; kk += 32) {
                    const double bv = (j < wc && kk < kl) ? __ldg(b + kk) : 0.0;
                    int dg[S];
                    make_digits<S, BETA>(bv, F, dg);
#pragma unroll
                    for (int s = 0; s < S; ++s)
                        *reinterpret_cast<uint16_t*>(dst + s * C_::planeB + (kk >> 3) * 128 + (kk & 7) * 2) =
                            digit_bits<FP16>(dg[s]);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                bool first_of_level[S + 2];
#pragma unroll
                for (int L = 0; L < S + 2; ++L) first_of_level[L] = (h0 == 0);
#pragma unroll
                for (int s = 1; s <= S; ++s) {
#pragma unroll
                    for (int t = 1; t <= S; ++t) {
                        if (s + t > S + 1) continue;
                        const int L = s + t;
                        const uint32_t dcol = tmem + (uint32_t)((L - 2) * kTN);
                        const uint32_t a_base = smem_u32(planeA + (s - 1) * C_::planeA);
                        const uint32_t b_base = smem_u32(planeB + (t - 1) * C_::planeB);
#pragma unroll
                        for (int q = 0; q < KS / 16; ++q) {
                            const uint64_t ad = make_desc(a_base + q * 256, C_::sbo);
                            const uint64_t bd = make_desc(b_base + q * 256, C_::sbo);
                            const uint32_t accum = first_of_level[L] ? 0u : 1u;
                            first_of_level[L] = false;
                            asm volatile(
                                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dcol),
                                "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
                        }
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                             : "memory");
            }
            // the digit planes are reused by the next sub-chunk: wait for the MMAs
            if (!mbar_wait(bar, phase)) failed = true;
            phase ^= 1;
            if (__syncthreads_or(failed)) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        }
        if (__syncthreads_or(failed)) {
            failed = true;
            break;
        }

        // ---- recombination of this chunk: TMEM levels -> exact binary64 ----
        {
            const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
#pragma unroll
            for (int g = 0; g < kTN / 16; ++g) {
                uint32_t v[S][16];
#pragma unroll
                for (int l = 0; l < S; ++l) {
                    const uint32_t ta = tmem + lane_base + (uint32_t)(l * kTN + g * 16);
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                        "[%16];\n"
                        : "=r"(v[l][0]), "=r"(v[l][1]), "=r"(v[l][2]), "=r"(v[l][3]), "=r"(v[l][4]), "=r"(v[l][5]),
                          "=r"(v[l][6]), "=r"(v[l][7]), "=r"(v[l][8]), "=r"(v[l][9]), "=r"(v[l][10]), "=r"(v[l][11]),
                          "=r"(v[l][12]), "=r"(v[l][13]), "=r"(v[l][14]), "=r"(v[l][15])
                        : "r"(ta));
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    const int j = g * 16 + jj;
                    long long I = 0;
#pragma unroll
                    for (int l = 0; l < S; ++l)   // level L = l + 2, weight 2^(beta (S - 1 - l))
                        I = (I << BETA) + (long long)__float2int_rn(__uint_as_float(v[l][jj]));
                    if (dump != nullptr && row_ok && j < wc) {
                        // exactness probe: the raw FP32 level sums of chunk c
#pragma unroll
                        for (int l = 0; l < S; ++l)
                            dump[(((size_t)c * S + l) * d.m + row) * d.n + (n0 + j)] = __uint_as_float(v[l][jj]);
                    }
                    acc[j] += scaled_int_to_double(I, E + s_F[j] - BETA * (S + 1));
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        }
        __syncthreads();   // TMEM reads and s_F use are done before the next chunk
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    }

    if (row_ok && !failed) {
#pragma unroll
        for (int j = 0; j < kTN; ++j)
            if (j < wc) d.C[(size_t)row + (size_t)(n0 + j) * (size_t)d.ldc] = acc[j];
    }
    if (failed) {
        // a wait expired: give the tensor-core work in flight one more bounded
        // wait before the TMEM it writes is released, and report the failure
        mbar_wait(bar, phase ^ 1);
        if (tid == 0) atomicExch(status, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
}

template <bool FP16, int S>
cudaError_t launch_t(const DevDesc* descs, const SItem* items, int n_items, int* status, float* dump,
                     cudaStream_t s) {
    const int smem = Cfg<FP16, S>::smem;
    cudaError_t e = cudaFuncSetAttribute(k_split<FP16, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (n_items <= 0) return cudaSuccess;
    k_split<FP16, S><<<n_items, kThreadsS, smem, s>>>(descs, items, status, dump);
    return cudaGetLastError();
}

cudaError_t launch_prec(int precision, const DevDesc* descs, const SItem* items, int n_items, int* status,
                        float* dump, cudaStream_t s) {
    switch (precision) {
        case LRB_PREC_SPLIT_BF16_S3: return launch_t<false, 3>(descs, items, n_items, status, dump, s);
        case LRB_PREC_SPLIT_BF16_S4: return launch_t<false, 4>(descs, items, n_items, status, dump, s);
        case LRB_PREC_SPLIT_FP16_S3: return launch_t<true, 3>(descs, items, n_items, status, dump, s);
        case LRB_PREC_SPLIT_FP16_S4: return launch_t<true, 4>(descs, items, n_items, status, dump, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

struct SplitPlan {
    int precision = 0;
    void* dmem = nullptr;
    DevDesc* d_descs = nullptr;
    SItem* d_items = nullptr;
    int* d_status = nullptr;
    int n_items = 0;
};

int chunk_len(int precision) {
    return (precision == LRB_PREC_SPLIT_FP16_S3 || precision == LRB_PREC_SPLIT_FP16_S4) ? 32 : 128;
}
int digit_count(int precision) {
    return (precision == LRB_PREC_SPLIT_BF16_S3 || precision == LRB_PREC_SPLIT_FP16_S3) ? 3 : 4;
}

lrb_status create(int device, int sms, const lrb_gemm_desc* descs, size_t count, int precision, SplitPlan** out,
                  lrb_plan_info* info) {
    (void)device;
    (void)sms;
    *out = nullptr;
    std::vector<SItem> items;
    for (size_t e = 0; e < count; ++e)
        for (int c0 = 0; c0 < descs[e].n; c0 += kTN)
            for (int r0 = 0; r0 < descs[e].m; r0 += kTM) items.push_back(SItem{(int32_t)e, r0, c0, 0});
    if (items.size() > 0x7fffffffull) {
        set_last_error("too many split-precision tiles");
        return LRB_ERR_INVALID;
    }
    SplitPlan* p = new SplitPlan();
    p->precision = precision;
    const size_t o_items = ((sizeof(DevDesc) * count + 255) / 256) * 256;
    const size_t o_status = o_items + ((sizeof(SItem) * std::max<size_t>(items.size(), 1) + 255) / 256) * 256;
    cudaError_t ce = cudaMalloc(&p->dmem, o_status + 256);
    if (ce != cudaSuccess) {
        delete p;
        set_last_error("split plan device memory");
        return LRB_ERR_NOMEM;
    }
    p->d_descs = (DevDesc*)p->dmem;
    p->d_items = (SItem*)((char*)p->dmem + o_items);
    p->d_status = (int*)((char*)p->dmem + o_status);
    p->n_items = (int)items.size();
    ce = cudaMemcpy(p->d_descs, descs, sizeof(DevDesc) * count, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess && !items.empty())
        ce = cudaMemcpy(p->d_items, items.data(), sizeof(SItem) * items.size(), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemset(p->d_status, 0, 256);
    if (ce != cudaSuccess) {
        cudaFree(p->dmem);
        delete p;
        set_last_error("split plan upload");
        return LRB_ERR_DEVICE;
    }
    info->items = p->n_items;
    info->groups = 1;
    info->grid = p->n_items;
    *out = p;
    return LRB_OK;
}

cudaError_t launch(SplitPlan* p, cudaStream_t s) {
    return launch_prec(p->precision, p->d_descs, p->d_items, p->n_items, p->d_status, nullptr, s);
}

cudaError_t launch_dump(SplitPlan* p, float* dump, cudaStream_t s) {
    return launch_prec(p->precision, p->d_descs, p->d_items, p->n_items, p->d_status, dump, s);
}

int read_status(SplitPlan* p, cudaStream_t s, int* value) {
    cudaError_t e = cudaMemcpyAsync(value, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? 0 : -1;
}

void destroy(SplitPlan* p) {
    if (!p) return;
    if (p->dmem) cudaFree(p->dmem);
    delete p;
}

}  // namespace split
}  // namespace lrb
