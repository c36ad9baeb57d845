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
//     L = s + t accumulate in one FP32 TMEM accumulator (BF16 S = 3: level
//     4's (2, 2) pair in a second one), exact because kc keeps every level
//     sum within 2^24 (BF16: beta 8, kc 64; FP16: beta 9, kc 32);
//   * per chunk the level sums are combined exactly as a 64-bit integer
//     I = sum_L P_L 2^(beta (S+1-L)) (|I| < 2^53), turned into the binary64
//     value I 2^(E_i + F_j - beta (S+1)) without rounding, and added to a
//     binary64 accumulator that starts from C.
//
// Kernel shape: a persistent CTA per SM (512 threads) walks its 128 x 64
// output tiles and their k-chunks as one pipeline.  Per chunk the threads
// load A (thread = tile row and a quarter of the chunk) and B into
// registers, compute the exponents (shared-memory exchange across the four
// quarters of a row; warp shuffles along B's columns) and write the digit
// planes into one of two shared-memory stages in the K-major, no-swizzle
// core-matrix layout (8 rows x 16 bytes per core matrix; LBO 128 bytes
// between core matrices along k, SBO = kc/8 * 128 bytes between 8-row
// groups); one thread issues tcgen05.mma (M 128, N 64, K 16) for every kept
// pair into one of two TMEM accumulator sets and commits to that stage's
// mbarrier; then the threads recombine the previous chunk from the other
// set.  Pre-sliced digit units (a plan's pre-passes) are copied into the
// stages with cp.async or, in mode 2, with bulk (TMA) copies on per-stage
// mbarriers.  Every wait is bounded (2 s): on expiry the kernel records an
// error in the plan's status word, drains its tensor-core work and copies
// (bounded), releases its TMEM and returns.
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
constexpr int kThreadsS = 512;
constexpr int kTmemCols = 512; // 2 sets x (up to) 4 accumulators x 64 columns
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s bound on any device-side wait


template <bool FP16, int S>
struct Cfg {
    static constexpr int beta = FP16 ? 9 : 8;
    static constexpr int kc = FP16 ? 32 : 64;      // k-chunk (one exponent per row / column)
    static constexpr int planeA = kTM * kc * 2;    // bytes per digit plane of A
    static constexpr int planeB = kTN * kc * 2;
    static constexpr int sbo = kc / 8 * 128;
    static constexpr int smem = 2 * S * (planeA + planeB);   // two stages
    static constexpr int unitB = S * planeB + 256;           // pre-sliced B chunk: planes + 64 exponents
    static constexpr int unitA = S * planeA + 512;           // pre-sliced A chunk: planes + 128 exponents
};

// One pre-sliced B chunk: columns [col0, col0 + 64) and rows [k0, k0 + kc)
// of entry `entry`'s B.  An A unit is rows [row0, row0 + 128) and columns
// [k0, k0 + kc) of A (the same struct, col0 read as row0).
struct BUnit {
    int32_t entry, col0, k0, pad;
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

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
    return t;
}

// Wait for the mbarrier phase with the given parity; gives up after about
// kWaitNs nanoseconds of wall time (the caller then reports an error).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const unsigned long long t0 = global_ns();
    for (long long i = 0;; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((i & 255) == 255 && global_ns() - t0 > kWaitNs) return false;
    }
}

// |a| bit pattern (sign cleared) -> E with 2^(E-1) <= |a| < 2^E (a != 0).
__device__ __forceinline__ int exp_of_bits(unsigned long long mag) {
    const int ef = (int)(mag >> 52);
    if (ef) return ef - 1022;
    return (64 - __clzll((long long)mag)) - 1074;   // subnormal
}

// Balanced digits of a given the chunk exponent E (see file comment).
// Z = RN_even(M 2^-sh) is formed with 64-bit integer shifts of the
// significand; the lowest digit comes off the 64-bit Z, the rest in 32-bit
// arithmetic (after one digit |Z| < 2^(beta (S-1) + 1) <= 2^28).
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
            Z = (long long)(M << (-sh));                     // subnormal rows only
        } else if (sh < 64) {
            const unsigned long long half = 1ull << (sh - 1);
            Z = (long long)((M + half - 1 + ((M >> sh) & 1ull)) >> sh);
        }
        if (bits >> 63) Z = -Z;
    }
    constexpr int base = 1 << BETA, h = 1 << (BETA - 1);
    // lowest digit from the 64-bit value (its low word suffices for the digit)
    const int d_last = (((int)(unsigned)Z + h) & (base - 1)) - h;
    d[S - 1] = d_last;
    int z = (int)((Z - d_last) >> BETA);
#pragma unroll
    for (int s = S - 2; s >= 1; --s) {
        const int dig = ((z + h) & (base - 1)) - h;
        d[s] = dig;
        z = (z - dig) >> BETA;
    }
    d[0] = z;
}

// 16-bit pattern of an integer digit |d| <= 2^(beta) (exact in either type).
// BF16: the float 1.5 * 2^23 + d, formed by an integer add to its bit
// pattern and the constant subtracted in float, is exactly d; its top 16 bits
// are the bf16 pattern.
template <bool FP16>
__device__ __forceinline__ uint16_t digit_bits(int d) {
    const float f = __int_as_float(0x4B400000 + d) - 12582912.0f;
    if constexpr (FP16) {
        return __half_as_ushort(__float2half_rn(f));
    } else {
        return (uint16_t)(__float_as_uint(f) >> 16);
    }
}

// Exact binary64 of I 2^X for |I| < 2^53, built from the bits: |I| shifted
// so its leading one sits at bit 52, plus (exponent - 1) << 52 (the leading
// one then completes the exponent field), plus the sign.
__device__ __forceinline__ double scaled_int_to_double(long long I, int X) {
    if (I == 0) return 0.0;
    const unsigned long long u = (unsigned long long)(I < 0 ? -I : I);
    const int lz = __clzll((long long)u);
    const int biased = 1023 + (63 - lz) + X;
    if (__builtin_expect(biased <= 0 || biased >= 2047, 0)) return ldexp((double)I, X);
    const unsigned long long b = (u << (lz - 11)) + ((unsigned long long)(biased - 1) << 52) +
                                 (I < 0 ? (1ull << 63) : 0ull);
    return __longlong_as_double((long long)b);
}

// ---- the 32-bit digit path (BF16, S = 3) ------------------------------------
// Key of a row of A within a chunk: the largest hi word of |a| (sign cleared),
// with bit 0 set when any lo word is nonzero.  The maximum's exponent field is
// key >> 20, so for key >= kKeyFastMin (a normal maximum of at least 2^-997)
// E = (key >> 20) - 1022, and key == 0 means every value is +-0; other keys
// (rows of values below 2^-997) take the exact 64-bit path.
constexpr uint32_t kKeyFastMin = 26u << 20;
__device__ __forceinline__ bool key_fast(uint32_t key) { return key == 0u || key >= kKeyFastMin; }
__device__ __forceinline__ int key_exponent(uint32_t key) { return key ? (int)(key >> 20) - 1022 : 0; }
// The right shift of an element with exponent field ef is key_shift(key) - ef
// (>= 7 in the row; a zero row shifts every element out).
__device__ __forceinline__ int key_shift(uint32_t key) { return key ? (int)(key >> 20) + 7 : (1 << 20); }

// x >> n for n in [0, 2^32), 0 once n >= 32 (PTX shr clamps the amount).
__device__ __forceinline__ uint32_t shr_clamped(uint32_t x, uint32_t n) {
    uint32_t r;
    asm("shr.b32 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(n));
    return r;
}

// The balanced digits of a (BF16, S = 3) for a row with key_fast(key), as
// floats whose top 16 bits are the BF16 patterns; the same digits as
// make_digits<3, 8>.  Z = RN_even(a 2^(24 - E)) on 32-bit words: W is a
// 31-bit window of the significand (the implicit one at bit 30), the lower
// 22 bits folded into W's lowest bit as a sticky bit; with sh = the window's
// right shift (>= 7, so the rounding position lies above the sticky bit),
// (W + 2^(sh-1) - 1 + bit sh of W) >> sh is the round-to-nearest-even of
// W / 2^sh and stays below 2^32; every shift clamps, so an element with sh >=
// 32 (below a quarter unit) gives 0.  Z + 0x8080 carries the two lower
// balanced digits into bytes (each digit + 128), d_1 is the rest; a digit d
// becomes the float 1.5 2^23 + d by placing it into that constant's bit
// pattern, minus the constant.  This part: the three patterns before the
// subtraction (d_1, then d_2 and d_3 offset by 128).
__device__ __forceinline__ void digit_patterns_bf16_s3(double a, int ksh, uint32_t& g1, uint32_t& g2, uint32_t& g3) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(a);
    const uint32_t h = (uint32_t)(bits >> 32), l = (uint32_t)bits;
    const uint32_t W = (__funnelshift_l(l, h, 11) >> 1) | 0x40000000u | min(l << 10, 1u);
    const uint32_t sh = (uint32_t)(ksh - (int)((h >> 20) & 0x7FFu));
    const uint32_t hm1 = shr_clamped(0x7FFFFFFFu, 32u - sh);   // 2^(sh-1) - 1 (0 once sh > 32)
    const uint32_t Z = shr_clamped(W + hm1 + (shr_clamped(W, sh) & 1u), sh);
    const int Zp = (int)Z * (((int)h >> 31) | 1) + 0x8080;
    g3 = __byte_perm((uint32_t)Zp, 0x4B400000u, 0x7650);
    g2 = __byte_perm((uint32_t)Zp, 0x4B400000u, 0x7651);
    g1 = (uint32_t)(0x4B400000 + (Zp >> 16));
}

// The digits of two elements a and b as float pairs (x: a, y: b), the
// constants subtracted by paired FP32 adds (one instruction per digit level
// for both elements, the same rounding as two scalar adds: all exact).
__device__ __forceinline__ void digits_bf16_s3_x2(double a, double b, int ksh, float2& f1, float2& f2, float2& f3) {
    uint32_t a1, a2, a3, b1, b2, b3;
    digit_patterns_bf16_s3(a, ksh, a1, a2, a3);
    digit_patterns_bf16_s3(b, ksh, b1, b2, b3);
    f3 = __fadd2_rn(make_float2(__uint_as_float(a3), __uint_as_float(b3)), make_float2(-12583040.0f, -12583040.0f));
    f2 = __fadd2_rn(make_float2(__uint_as_float(a2), __uint_as_float(b2)), make_float2(-12583040.0f, -12583040.0f));
    f1 = __fadd2_rn(make_float2(__uint_as_float(a1), __uint_as_float(b1)), make_float2(-12582912.0f, -12582912.0f));
}

// TMEM accumulators per chunk: one per level L = 2 .. S + 1, except that
// BF16 S = 3 gives the (2, 2) pair of level 4 one of its own.  Level 4 can
// reach 5 2^20 there, beyond the 2^22 of the conversion below; its parts
// (1, 3) + (3, 1) and (2, 2) stay within 2^22 and 2^20.
template <bool FP16, int S>
__host__ __device__ constexpr int n_acc() { return (!FP16 && S == 3) ? S + 1 : S; }

// The accumulator of digit pair (s, t).
template <bool FP16, int S>
__host__ __device__ constexpr int acc_of(int s, int t) {
    return (!FP16 && S == 3 && s == 2 && t == 2) ? S : s + t - 2;
}

// Largest |P| one k-chunk can produce in accumulator g (kc times its kept
// pairs' largest digit products; max|d_1| = 2^beta, max|d_s| = 2^(beta-1)).
template <bool FP16, int S>
__host__ __device__ constexpr long long acc_bound_c(int g) {
    const int beta = FP16 ? 9 : 8, kc = FP16 ? 32 : 64;
    long long b = 0;
    for (int s = 1; s <= S; ++s)
        for (int t = 1; t <= S; ++t)
            if (s + t <= S + 1 && acc_of<FP16, S>(s, t) == g)
                b += (long long)(s == 1 ? 1 << beta : 1 << (beta - 1)) * (t == 1 ? 1 << beta : 1 << (beta - 1));
    return b * kc;
}

// Accumulator g as an integer.  Where |P| <= 2^22 the float P + 1.5 2^23 is
// exact and its bit pattern is 0x4B400000 + P (an FP32 add, no conversion
// instruction); larger bounds convert.  ADDED: v already holds P + 1.5 2^23
// (the caller added the constant to pairs of accumulators at once).
template <bool FP16, int S, bool ADDED = false>
__device__ __forceinline__ int acc_value(uint32_t v, int g) {
    if (acc_bound_c<FP16, S>(g) <= (1ll << 22)) {
        if constexpr (ADDED) return (int)v - 0x4B400000;
        return __float_as_int(__uint_as_float(v) + 12582912.0f) - 0x4B400000;
    }
    return __float2int_rn(__uint_as_float(v));
}

// Every accumulator of the preset converts with the FP32 add.
template <bool FP16, int S>
__host__ __device__ constexpr bool all_acc_magic() {
    for (int g = 0; g < n_acc<FP16, S>(); ++g)
        if (acc_bound_c<FP16, S>(g) > (1ll << 22)) return false;
    return true;
}

// I = sum_L P_L 2^(beta (S + 1 - L)) of one output (accumulator g in v[g];
// level L = g + 2 for g < S).  BF16: the two lowest levels combine in 32 bits
// (|P_L 2^8 + P_L'| < 2^31), as do the two highest for S = 4, and one wide
// multiply-add joins them.
template <bool FP16, int S, int RC, bool ADDED = false>
__device__ __forceinline__ long long level_integer(const uint32_t (&v)[n_acc<FP16, S>()][RC], int jj) {
    if constexpr (!FP16 && S == 3) {
        const int hi = acc_value<FP16, S, ADDED>(v[0][jj], 0);
        const int p4 = acc_value<FP16, S, ADDED>(v[2][jj], 2) + acc_value<FP16, S, ADDED>(v[3][jj], 3);
        const int lo = acc_value<FP16, S, ADDED>(v[1][jj], 1) * 256 + p4;
        return (long long)hi * 65536 + lo;
    } else if constexpr (!FP16 && S == 4) {
        const int hi = acc_value<FP16, S>(v[0][jj], 0) * 256 + acc_value<FP16, S>(v[1][jj], 1);
        const int lo = acc_value<FP16, S>(v[2][jj], 2) * 256 + acc_value<FP16, S>(v[3][jj], 3);
        return (long long)hi * 65536 + lo;
    } else {
        constexpr int BETA = FP16 ? 9 : 8;
        long long I = 0;
#pragma unroll
        for (int l = 0; l < S; ++l) I = I * (1ll << BETA) + acc_value<FP16, S>(v[l][jj], l);
        return I;
    }
}

// The B part of one chunk, by 512 threads: column exponents F (to F_out[64])
// and the S digit planes (to planes, in the core-matrix layout the MMA reads).
// A column's kc values are split over kc / 8 neighbouring lanes, each with 8
// consecutive k values: its column maximum by shuffles among them, and each
// plane's 8 digits of one column form one 16-byte core-matrix row, written
// with one store.  Used by the pre-pass, which writes to global memory; the
// digits come from the same function as the in-kernel slicing, so they are
// the same whichever runs.
template <bool FP16, int S>
__device__ __forceinline__ void slice_b_chunk(const DevDesc& d, int n0, int k0, int warp, int lane,
                                              uint8_t* planes, int* F_out) {
    using C_ = Cfg<FP16, S>;
    constexpr int BETA = C_::beta, KC = C_::kc;
    constexpr int LPC = KC / 8;        // lanes per column
    constexpr int CPW = 32 / LPC;      // columns per warp
    if (warp >= kTN / CPW) return;     // FP16 (kc 32): half the warps cover the 64 columns
    const int j = warp * CPW + lane / LPC, sub = lane % LPC;
    const int kcl = min(KC, d.k - k0);
    const int wc = min(kTN, d.n - n0);
    double bv[8];
    unsigned long long mx = 0;
    const double* bp = d.B + (size_t)(k0 + 8 * sub) + (size_t)(n0 + j) * (size_t)d.ldb;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        bv[i] = (j < wc && 8 * sub + i < kcl) ? __ldg(bp + i) : 0.0;
        const unsigned long long v = (unsigned long long)__double_as_longlong(bv[i]) & 0x7FFFFFFFFFFFFFFFull;
        mx = v > mx ? v : mx;
    }
#pragma unroll
    for (int o = LPC / 2; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = w > mx ? w : mx;
    }
    const int F = mx ? exp_of_bits(mx) : 0;
    if (sub == 0) F_out[j] = F;
    uint32_t packed[S][4];
    bool fast = false;
    if constexpr (!FP16 && S == 3) {
        // the 32-bit digit path of the in-kernel slicing of A, for a column
        // whose key (largest high word, bit 0 set when any low word is
        // nonzero; the same over the column's lanes) allows it: the same
        // digits as the 64-bit path, in fewer instructions
        uint32_t key = 0, lo = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const unsigned long long bb = (unsigned long long)__double_as_longlong(bv[i]);
            key = max(key, (uint32_t)(bb >> 32) & 0x7FFFFFFFu);
            lo |= (uint32_t)bb;
        }
        key |= lo != 0u ? 1u : 0u;
#pragma unroll
        for (int o = LPC / 2; o > 0; o >>= 1) key = max(key, __shfl_xor_sync(0xffffffffu, key, o));
        fast = key_fast(key);
        if (fast) {
            const int ksh = key_shift(key);
#pragma unroll
            for (int p = 0; p < 8; p += 2) {
                float2 f1, f2, f3;
                digits_bf16_s3_x2(bv[p], bv[p + 1], ksh, f1, f2, f3);
                packed[0][p >> 1] = __byte_perm(__float_as_uint(f1.x), __float_as_uint(f1.y), 0x7632);
                packed[1][p >> 1] = __byte_perm(__float_as_uint(f2.x), __float_as_uint(f2.y), 0x7632);
                packed[2][p >> 1] = __byte_perm(__float_as_uint(f3.x), __float_as_uint(f3.y), 0x7632);
            }
        }
    }
    if (!fast) {
#pragma unroll
        for (int p = 0; p < 8; p += 2) {
            int d0[S], d1[S];
            make_digits<S, BETA>(bv[p], F, d0);
            make_digits<S, BETA>(bv[p + 1], F, d1);
#pragma unroll
            for (int s2 = 0; s2 < S; ++s2)
                packed[s2][p >> 1] = (uint32_t)digit_bits<FP16>(d0[s2]) | ((uint32_t)digit_bits<FP16>(d1[s2]) << 16);
        }
    }
    uint8_t* dst = planes + (j >> 3) * C_::sbo + (j & 7) * 16 + sub * 128;
#pragma unroll
    for (int s2 = 0; s2 < S; ++s2)
        *reinterpret_cast<uint4*>(dst + s2 * C_::planeB) =
            make_uint4(packed[s2][0], packed[s2][1], packed[s2][2], packed[s2][3]);
}

// Pre-pass: one 512-thread CTA per B unit (entry, 64-column tile, k-chunk);
// at most 40 registers, so three CTAs share an SM (measured: as fast or
// faster than two at 46 registers).
// Every 128-row tile of an entry uses the same B chunks; slicing them once
// here instead of once per row tile removes the repeated integer work.
template <bool FP16, int S>
__global__ void __launch_bounds__(kThreadsS, 3) k_slice_b(const DevDesc* __restrict__ descs,
                                                       const BUnit* __restrict__ units, uint8_t* __restrict__ out) {
    using C_ = Cfg<FP16, S>;
    const BUnit u = units[blockIdx.x];
    const DevDesc d = descs[u.entry];
    uint8_t* dst = out + (size_t)blockIdx.x * C_::unitB;
    slice_b_chunk<FP16, S>(d, u.col0, u.k0, threadIdx.x >> 5, threadIdx.x & 31, dst,
                           reinterpret_cast<int*>(dst + S * C_::planeB));
}

// Pre-pass for entries with several 64-column tiles (each 128-row tile of A
// would otherwise be sliced once per column tile): one 512-thread CTA per A
// unit; thread (row 32 (w % 4) + lane, quarter w / 4 of the chunk) as in the
// main kernel, row exponents through shared memory, digit planes and the 128
// exponents written to global memory.
template <bool FP16, int S>
__global__ void __launch_bounds__(kThreadsS) k_slice_a(const DevDesc* __restrict__ descs,
                                                       const BUnit* __restrict__ units, uint8_t* __restrict__ out) {
    using C_ = Cfg<FP16, S>;
    constexpr int BETA = C_::beta, KC = C_::kc, QC = KC / 4;
    __shared__ unsigned long long s_rmax[4][kTM];
    __shared__ uint32_t s_rkey[4][kTM];
    const BUnit u = units[blockIdx.x];
    const DevDesc d = descs[u.entry];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rloc = 32 * (warp & 3) + lane, q = warp >> 2;
    const int row = u.col0 + rloc, k0 = u.k0;
    const int kcl = min(KC, d.k - k0);
    uint8_t* dst0 = out + (size_t)blockIdx.x * C_::unitA;
    double av[QC];
    {
        const double* ap = d.A + (size_t)row + (size_t)(k0 + q * QC) * (size_t)d.lda;
        const int ncol = row < d.m ? min(QC, kcl - q * QC) : 0;
#pragma unroll
        for (int p = 0; p < QC; ++p) {
            av[p] = p < ncol ? __ldg(ap) : 0.0;
            ap += d.lda;
        }
    }
    unsigned long long mx = 0;
#pragma unroll
    for (int p = 0; p < QC; ++p) {
        const unsigned long long v = (unsigned long long)__double_as_longlong(av[p]) & 0x7FFFFFFFFFFFFFFFull;
        mx = v > mx ? v : mx;
    }
    s_rmax[q][rloc] = mx;
    constexpr bool KEYED = !FP16 && S == 3;   // the 32-bit digit path, as in the kernel's own slicing
    if constexpr (KEYED) {
        uint32_t hmx = 0, lo = 0;
#pragma unroll
        for (int p = 0; p < QC; ++p) {
            const unsigned long long bb = (unsigned long long)__double_as_longlong(av[p]);
            hmx = max(hmx, (uint32_t)(bb >> 32) & 0x7FFFFFFFu);
            lo |= (uint32_t)bb;
        }
        s_rkey[q][rloc] = hmx | (lo != 0u ? 1u : 0u);
    }
    __syncthreads();
    mx = s_rmax[0][rloc];
#pragma unroll
    for (int qq = 1; qq < 4; ++qq) mx = s_rmax[qq][rloc] > mx ? s_rmax[qq][rloc] : mx;
    const int E = mx ? exp_of_bits(mx) : 0;
    if (q == 0) reinterpret_cast<int*>(dst0 + S * C_::planeA)[rloc] = E;
    // a row whose key allows it (the same for the row's four quarters) takes the
    // 32-bit digit path: the same digits in fewer instructions
    bool fast = false;
    int ksh = 0;
    if constexpr (KEYED) {
        const uint32_t key = max(max(s_rkey[0][rloc], s_rkey[1][rloc]), max(s_rkey[2][rloc], s_rkey[3][rloc]));
        fast = key_fast(key);
        ksh = key_shift(key);
    }
    uint8_t* dst = dst0 + (rloc >> 3) * C_::sbo + (rloc & 7) * 16 + (q * QC / 8) * 128;
#pragma unroll
    for (int g = 0; g < QC / 8; ++g) {
        uint32_t packed[S][4];
        if (fast) {
            if constexpr (KEYED) {
#pragma unroll
                for (int p = 0; p < 8; p += 2) {
                    float2 f1, f2, f3;
                    digits_bf16_s3_x2(av[8 * g + p], av[8 * g + p + 1], ksh, f1, f2, f3);
                    packed[0][p >> 1] = __byte_perm(__float_as_uint(f1.x), __float_as_uint(f1.y), 0x7632);
                    packed[1][p >> 1] = __byte_perm(__float_as_uint(f2.x), __float_as_uint(f2.y), 0x7632);
                    packed[2][p >> 1] = __byte_perm(__float_as_uint(f3.x), __float_as_uint(f3.y), 0x7632);
                }
            }
        } else {
#pragma unroll
            for (int p = 0; p < 8; p += 2) {
                int d0[S], d1[S];
                make_digits<S, BETA>(av[8 * g + p], E, d0);
                make_digits<S, BETA>(av[8 * g + p + 1], E, d1);
#pragma unroll
                for (int s2 = 0; s2 < S; ++s2)
                    packed[s2][p >> 1] = (uint32_t)digit_bits<FP16>(d0[s2]) | ((uint32_t)digit_bits<FP16>(d1[s2]) << 16);
            }
        }
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2)
            *reinterpret_cast<uint4*>(dst + s2 * C_::planeA + g * 128) =
                make_uint4(packed[s2][0], packed[s2][1], packed[s2][2], packed[s2][3]);
    }
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem_dst)), "l"(src) : "memory");
}

// One bulk (TMA) copy of `bytes` (a multiple of 16, both addresses 16-byte
// aligned) from global to this CTA's shared memory, completing on mbarrier
// `bar` (the caller has announced the bytes with expect_tx).
__device__ __forceinline__ void bulk_copy(void* smem_dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(smem_dst)),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// One CTA per SM, 512 threads, tiles taken round-robin (tile = 128 x 64
// outputs).  The k-chunks of all of a CTA's tiles form one pipeline: while
// the tensor cores run chunk i (digit planes and TMEM accumulator set i&1),
// the threads recombine chunk i-1 from the other TMEM set.  The operands of
// chunk i+1 are loaded into registers as soon as chunk i's digits are in
// shared memory, so their latency hides behind chunk i's tensor-core issue
// and chunk i-1's recombination.  Thread t: row 32 (w % 4) + lane of the tile
// (w = warp, = its TMEM lane), quarter q = w / 4 of the chunk's columns for
// slicing and of the tile's 64 output columns for recombination.
template <bool FP16, int S, int MODE>
__global__ void __launch_bounds__(kThreadsS, 1) k_split(const STile* __restrict__ tiles, int n_items,
                                                         int* __restrict__ status, float* __restrict__ dump,
                                                         int test_stall, const uint8_t* __restrict__ bunits,
                                                         const long long* __restrict__ bfirst,
                                                         const uint8_t* __restrict__ aunits,
                                                         const long long* __restrict__ afirst) {
    // MODE 0: the kernel slices A and B (serving waves).  MODE 1: B comes
    // pre-sliced (k_slice_b), unit of (entry, column tile ct, chunk c) =
    // bfirst[entry] + ct * chunks + c.  MODE 2: A too (k_slice_a), unit
    // afirst[entry] + row tile * chunks + c (entries with several column tiles).
    constexpr bool PRE = MODE >= 1;
    constexpr bool preA = MODE == 2;
    // A's digits on the 32-bit path (BF16, S = 3; MODE 1, the T-form path:
    // MODE 0 also slices B and would spill registers with both paths compiled)
    constexpr bool FAST = !FP16 && S == 3 && MODE == 1;
    // FAST also loads the next chunk's A while the tensor cores and the
    // recombination run (the other paths spill registers with that)
    constexpr bool PRELOAD = FAST;
    using C_ = Cfg<FP16, S>;
    constexpr int BETA = C_::beta, KC = C_::kc;
    constexpr int QC = KC / 4;            // chunk columns of A per thread
    constexpr int KB = KC / 32;           // k values of B per lane and column
    constexpr int NACC = n_acc<FP16, S>();   // TMEM accumulators (64 columns each) per stage
    static_assert(2 * NACC * kTN <= kTmemCols, "two stages of accumulators must fit the TMEM allocation");
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ unsigned long long s_rmax[4][kTM];
    __shared__ uint32_t s_rkey[4][kTM];
    // row and column exponents of the last three chunks (slot = chunk index
    // mod 3): a thread may write chunk i + 1's while another still reads chunk
    // i - 1's in its recombination; one that writes chunk i + 2's has passed
    // the barrier that every thread reaches only after that recombination
    __shared__ __align__(16) int s_E[3][kTM];
    __shared__ __align__(16) int s_F[3][kTN];
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ __align__(8) uint64_t s_ubar[2];   // pre-sliced units copied into each stage (bulk copies)
    __shared__ __align__(8) uint64_t s_never;   // test_stall: a barrier nothing arrives on
    // the records of the CTA's tiles in a ring of eight: the record three
    // tiles ahead is copied while a tile starts, so no tile waits on a global
    // load of its own record, and mode 2 (one chunk per tile in the usual
    // case) need not wait for the copy it has just issued.  Slot ti & 7 holds
    // tile ti.  A thread that starts tile ti + 1 (and writes slot (ti + 4) & 7)
    // may meet threads still in tile ti, which read slots ti & 7 and
    // (ti + 1) & 7, never one still in tile ti - 1.
    __shared__ __align__(16) STile s_tile[8];
    __shared__ uint32_t s_tmem;
    // a recombination wait expired in an iteration of this parity: set before
    // the next iteration's issue barrier, read by every thread after it (a
    // thread still reading iteration i's slot cannot meet a write to it from
    // iteration i + 2, which needs that barrier passed)
    __shared__ int s_fail[2];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rloc = 32 * (warp & 3) + lane;   // tile row (TMEM lane)
    const int q = warp >> 2;                   // quarter

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&s_bar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&s_bar[1])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&s_never)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&s_ubar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&s_ubar[1])));
        s_fail[0] = s_fail[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = s_tmem;
    const uint32_t idesc = make_idesc<FP16>();
    bool failed = false;

    // the chunk whose MMAs are in flight (recombined one iteration later)
    struct Prev {
        double* C;          // the tile's entry: C, its extent and leading dimension
        int m, n, ldc;
        int row0, col0, c, stage, slot;
        bool last;
    } prev{};
    bool have_prev = false;
    double acc[16];

    // C of the thread's row and 16 columns: the column pointer advances by
    // ldc; a tile that covers all 16 columns (the usual case) skips the
    // per-column test.  C is read once and written once, so both go with the
    // streaming cache hint (O-form 0.3 % faster)
    auto load_c0 = [&](const DevDesc& d, int row0, int col0) {
        const int row = row0 + rloc, c1 = col0 + 16 * q;
        const double* cp = d.C + (size_t)row + (size_t)c1 * (size_t)d.ldc;
        const size_t ld = (size_t)d.ldc;
        if (row < d.m && c1 + 16 <= d.n) {
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) acc[jj] = __ldcs(cp + jj * ld);
        } else {
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) acc[jj] = (row < d.m && c1 + jj < d.n) ? __ldcs(cp + jj * ld) : 0.0;
        }
    };

    // The operands this thread slices for one chunk, in registers: A row
    // m0 + rloc, chunk columns [k0 + q QC, k0 + q QC + QC); B columns 4 w ..
    // 4 w + 3 of the tile, k values lane + 32 h.  Zero outside the entry.
    double av[preA ? 1 : QC];
    double bv[PRE ? 1 : 4][KB];
    auto load_chunk = [&](const DevDesc& d, int m0, int n0, int k0) {
        const int kcl = min(KC, d.k - k0);
        if constexpr (!preA) {
            const int row = m0 + rloc;
            const double* ap = d.A + (size_t)row + (size_t)(k0 + q * QC) * (size_t)d.lda;
            const int ncol = row < d.m ? min(QC, kcl - q * QC) : 0;   // valid columns of this quarter
#pragma unroll
            for (int p = 0; p < QC; ++p) {
                av[p] = p < ncol ? __ldg(ap) : 0.0;
                ap += d.lda;
            }
        }
        if constexpr (!PRE) {
            const int wc = min(kTN, d.n - n0);
#pragma unroll
            for (int jc = 0; jc < 4; ++jc) {
                const int j = 4 * warp + jc;
#pragma unroll
                for (int h = 0; h < KB; ++h) {
                    const int kk = lane + 32 * h;
                    bv[jc][h] = (j < wc && kk < kcl)
                                    ? __ldg(d.B + (size_t)(k0 + kk) + (size_t)(n0 + j) * (size_t)d.ldb)
                                    : 0.0;
                }
            }
        }
    };

    // recombine `prev` into acc (its MMAs committed to s_bar[prev.stage])
    auto recombine = [&](uint32_t parity) -> bool {
        // warp-uniform decision before the warp-collective TMEM loads
        if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&s_bar[prev.stage]), parity))) return false;
        if (test_stall && !__all_sync(0xffffffffu, mbar_wait(smem_u32(&s_never), 0))) return false;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
        const int E = s_E[prev.slot][rloc];
        const int row = prev.row0 + rloc;
        // the thread's 16 output columns in groups of RC (MODE 1 holds the next
        // chunk's operands in registers meanwhile, so it loads 4 at a time)
        constexpr int RC = PRELOAD ? 4 : 8;
#pragma unroll
        for (int grp = 0; grp < 16 / RC; ++grp) {
            uint32_t v[NACC][RC];
#pragma unroll
            for (int l = 0; l < NACC; ++l) {
                const uint32_t ta = tmem + lane_base + (uint32_t)(prev.stage * NACC * kTN + l * kTN + 16 * q + RC * grp);
                if constexpr (RC == 8) {
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                                 : "=r"(v[l][0]), "=r"(v[l][1]), "=r"(v[l][2]), "=r"(v[l][3]), "=r"(v[l][4]),
                                   "=r"(v[l][5]), "=r"(v[l][6]), "=r"(v[l][7])
                                 : "r"(ta));
                } else {
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n"
                                 : "=r"(v[l][0]), "=r"(v[l][1]), "=r"(v[l][2]), "=r"(v[l][3])
                                 : "r"(ta));
                }
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            if (dump != nullptr) {   // the diagnostic (a uniform branch, outside the per-output work)
#pragma unroll
                for (int jj = 0; jj < RC; ++jj) {
                    const int j = 16 * q + RC * grp + jj;
                    if (row < prev.m && prev.col0 + j < prev.n) {
#pragma unroll
                        for (int l = 0; l < S; ++l) {
                            // a level's parts are integers below 2^24 in sum: exact
                            float val = __uint_as_float(v[l][jj]);
                            if (NACC > S && l == S - 1) val += __uint_as_float(v[S][jj]);
                            dump[(((size_t)prev.c * S + l) * prev.m + row) * prev.n + (prev.col0 + j)] = val;
                        }
                    }
                }
            }
            // every accumulator's FP32 add for two columns at a time (the
            // loaded registers of neighbouring columns are adjacent).  Mode 1
            // only: measured 0.5 % faster there and 1.7 % slower in mode 2
            constexpr bool PAIRED = MODE == 1 && all_acc_magic<FP16, S>();
            if constexpr (PAIRED) {
#pragma unroll
                for (int l = 0; l < NACC; ++l) {
#pragma unroll
                    for (int jj = 0; jj < RC; jj += 2) {
                        const float2 w = __fadd2_rn(make_float2(__uint_as_float(v[l][jj]), __uint_as_float(v[l][jj + 1])),
                                                    make_float2(12582912.0f, 12582912.0f));
                        v[l][jj] = __float_as_uint(w.x);
                        v[l][jj + 1] = __float_as_uint(w.y);
                    }
                }
            }
            // the group's column exponents (E + F_j - beta (S + 1) per column)
            int Fx[RC];
#pragma unroll
            for (int jj = 0; jj < RC; jj += 4) {
                const int4 f4 = *reinterpret_cast<const int4*>(&s_F[prev.slot][16 * q + RC * grp + jj]);
                Fx[jj] = f4.x;
                Fx[jj + 1] = f4.y;
                Fx[jj + 2] = f4.z;
                Fx[jj + 3] = f4.w;
            }
#pragma unroll
            for (int jj = 0; jj < RC; ++jj) {
                // level L = l + 2 has weight 2^(beta (S - 1 - l))
                const long long I = level_integer<FP16, S, RC, PAIRED>(v, jj);
                // the exact binary64 value I 2^X (built from bits with integer
                // instructions), then one binary64 add.  (Forming it on the FP64
                // pipe instead -- 1.5 2^52 + I from bits, minus 1.5 2^52, one FMA
                // by 2^X -- measured slower: the FP64 pipe, not the integer ALU,
                // then limits.)
                acc[RC * grp + jj] += scaled_int_to_double(I, E + Fx[jj] - BETA * (S + 1));
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        return true;
    };

    auto store_prev = [&]() {
        const int row = prev.row0 + rloc, c1 = prev.col0 + 16 * q;
        double* cp = prev.C + (size_t)row + (size_t)c1 * (size_t)prev.ldc;
        const size_t ld = (size_t)prev.ldc;
        if (row < prev.m) {
            if (c1 + 16 <= prev.n) {
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) __stcs(cp + jj * ld, acc[jj]);
            } else {
#pragma unroll
                for (int jj = 0; jj < 16; ++jj)
                    if (c1 + jj < prev.n) __stcs(cp + jj * ld, acc[jj]);
            }
        }
    };

    // Pre-sliced digit units of chunk cc of tile (entry, r0, c0) into stage stg
    // (planes) and exponent slot sl: B's planes and column exponents, and
    // (MODE 2) A's planes and row exponents.
    // Copied by every thread in 16-byte pieces with cp.async (one commit
    // group), or, with BULK (mode 2 with at most 80 KB of units per stage:
    // BF16 S = 3 and the FP16 presets), by one thread as bulk (TMA) copies that
    // complete on the stage's unit barrier s_ubar[stg].  Measured: bulk copies
    // 2-3 % faster in mode 2 with those units, 3 % slower with BF16 S = 4's
    // 99 KB, and 1.4 % slower in mode 1, where the per-thread copies overlap
    // the slicing of A.  With BULK every thread counts the copies per stage
    // (ucount), which gives the phase to wait for.  A stage is refilled only
    // after the tensor-core work that read it has completed, and every thread
    // has waited for the previous fill before that work was issued, so a
    // phase is never reused early.
    constexpr bool BULK = MODE == 2 && C_::unitA + C_::unitB <= 80 * 1024;
    uint32_t ucount[2] = {0u, 0u};
    auto copy_units = [&](int entry, int r0, int c0, int nch_e, int cc, int stg, int sl) {
        if constexpr (!BULK) {
            uint8_t* pa = smem + stg * (S * (C_::planeA + C_::planeB));
            uint8_t* pb = pa + S * C_::planeA;
            if constexpr (MODE == 2) {
                const uint8_t* src = aunits + (size_t)(afirst[entry] + (long long)(r0 / kTM) * nch_e + cc) * C_::unitA;
                for (int o = 16 * tid; o < S * C_::planeA; o += 16 * kThreadsS) cp_async16(pa + o, src + o);
                if (tid < kTM / 4) cp_async16(&s_E[sl][4 * tid], src + S * C_::planeA + 16 * tid);
            }
            const uint8_t* src = bunits + (size_t)(bfirst[entry] + (long long)(c0 / kTN) * nch_e + cc) * C_::unitB;
            for (int o = 16 * tid; o < S * C_::planeB; o += 16 * kThreadsS) cp_async16(pb + o, src + o);
            if (tid < kTN / 4) cp_async16(&s_F[sl][4 * tid], src + S * C_::planeB + 16 * tid);
            asm volatile("cp.async.commit_group;\n" ::: "memory");
        } else {
            if (tid == 0) {
                uint8_t* pa = smem + stg * (S * (C_::planeA + C_::planeB));
                uint8_t* pb = pa + S * C_::planeA;
                const uint32_t bar = smem_u32(&s_ubar[stg]);
                constexpr uint32_t bytes = (MODE == 2 ? (uint32_t)C_::unitA : 0u) + (uint32_t)C_::unitB;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
                if constexpr (MODE == 2) {
                    const uint8_t* src = aunits + (size_t)(afirst[entry] + (long long)(r0 / kTM) * nch_e + cc) * C_::unitA;
                    bulk_copy(pa, src, S * C_::planeA, bar);
                    bulk_copy(&s_E[sl][0], src + S * C_::planeA, 4 * kTM, bar);
                }
                const uint8_t* src = bunits + (size_t)(bfirst[entry] + (long long)(c0 / kTN) * nch_e + cc) * C_::unitB;
                bulk_copy(pb, src, S * C_::planeB, bar);
                bulk_copy(&s_F[sl][0], src + S * C_::planeB, 4 * kTN, bar);
            }
            ++ucount[stg];
        }
    };

    int iter = 0;
    int slot = 0;             // iter mod 3: the chunk's exponent slot
    int last_commit = -1;     // iteration of the most recent tensor-core commit
    int t = blockIdx.x;
    if (tid < 12) {   // the first three records, synchronously
        const int tt = t + (tid >> 2) * (int)gridDim.x;
        if (tt < n_items)
            reinterpret_cast<uint4*>(&s_tile[tid >> 2])[tid & 3] = reinterpret_cast<const uint4*>(tiles + tt)[tid & 3];
    }
    __syncthreads();
    if (t < n_items) {
        const STile& r0 = s_tile[0];
        load_c0(r0.d, r0.row0, r0.col0);
        if constexpr (PRELOAD) load_chunk(r0.d, r0.row0, r0.col0, 0);
    }
    int ti = 0;   // index of the CTA's current tile (its record is s_tile[ti & 7])
    while (t < n_items) {
        const STile& cur = s_tile[ti & 7];
        const DevDesc d = cur.d;
        const int entry = cur.entry;
        const int m0 = cur.row0, n0 = cur.col0;
        const int nch = (d.k + KC - 1) / KC;
        const int tn = t + gridDim.x;
        const STile& nxt = s_tile[(ti + 1) & 7];   // valid when tn < n_items
        {
            // the record three tiles ahead into the ring slot tile ti - 5 used
            // (one commit group; complete before the tensor-core issue of this
            // tile's second chunk or of the next tile's first, and visible to
            // every thread after the barrier there, so before tile ti + 2 reads
            // it as its next tile)
            const int t3 = tn + 2 * (int)gridDim.x;
            if (tid < 4 && t3 < n_items) cp_async16(reinterpret_cast<uint4*>(&s_tile[(ti + 3) & 7]) + tid,
                                                    reinterpret_cast<const uint4*>(tiles + t3) + tid);
            asm volatile("cp.async.commit_group;\n" ::: "memory");
            // the CTA's next tile into L2 while this one runs: its C (one
            // 128-byte line of 16 rows per thread) and, when pre-sliced, its
            // first chunk's digit units
            if (tn < n_items) {
                const STile& nx = nxt;
                const DevDesc dn = nx.d;
                const int jj = tid >> 3, r = nx.row0 + 16 * (tid & 7);
                if (jj < kTN && nx.col0 + jj < dn.n && r < dn.m)
                    asm volatile("prefetch.global.L2 [%0];\n" ::"l"(dn.C + (size_t)r + (size_t)(nx.col0 + jj) * (size_t)dn.ldc));
                if constexpr (MODE >= 1) {
                    const int nchn = (dn.k + KC - 1) / KC;
                    const uint8_t* ub = bunits + (size_t)(bfirst[nx.entry] + (long long)(nx.col0 / kTN) * nchn) * C_::unitB;
                    for (int o = 128 * tid; o < C_::unitB; o += 128 * kThreadsS)
                        asm volatile("prefetch.global.L2 [%0];\n" ::"l"(ub + o));
                    if constexpr (MODE == 2) {
                        const uint8_t* ua =
                            aunits + (size_t)(afirst[nx.entry] + (long long)(nx.row0 / kTM) * nchn) * C_::unitA;
                        for (int o = 128 * tid; o < C_::unitA; o += 128 * kThreadsS)
                            asm volatile("prefetch.global.L2 [%0];\n" ::"l"(ua + o));
                    }
                }
            }
        }
        for (int c = 0; c < nch; ++c, ++iter, slot = slot == 2 ? 0 : slot + 1) {
            const int stage = iter & 1;
            const int slot_next = slot == 2 ? 0 : slot + 1;
            const int k0 = c * KC;
            uint8_t* planeA = smem + stage * (S * (C_::planeA + C_::planeB));
            uint8_t* planeB = planeA + S * C_::planeA;
            // (0) pre-sliced units.  MODE 1 copies this chunk's B here, where the
            // copy overlaps the slicing of A; MODE 2 (nothing else to overlap)
            // copies the next chunk's units one iteration ahead (step 5), so
            // only the CTA's first chunk copies its own here.
            if constexpr (PRE) {
                if (MODE == 1 || iter == 0) copy_units(entry, m0, n0, nch, c, stage, slot);
            }
            if constexpr (!PRELOAD && !preA) load_chunk(d, m0, n0, k0);
            // (1) a later chunk into L2 (with PRELOAD: the one after the next,
            // whose loads step 3b issues; else the next): one 128-byte line per
            // thread (A: 16 rows of one column; B: 16 k of one column),
            // in-bounds addresses only
            if (c + (PRELOAD ? 2 : 1) < nch) {
                const int kn = k0 + (PRELOAD ? 2 : 1) * KC;
                const int kk = tid >> 3, r = m0 + 16 * (tid & 7);
                if (!preA && kk < KC && kn + kk < d.k && r < d.m)
                    asm volatile("prefetch.global.L2 [%0];\n" ::"l"(d.A + (size_t)r + (size_t)(kn + kk) * (size_t)d.lda));
                if (!PRE && tid < kTN * (KC / 16)) {
                    const int j = tid / (KC / 16), kb = kn + 16 * (tid % (KC / 16));
                    if (j < min(kTN, d.n - n0) && kb < d.k)
                        asm volatile("prefetch.global.L2 [%0];\n" ::"l"(d.B + (size_t)kb + (size_t)(n0 + j) * (size_t)d.ldb));
                }
            }
            // (2) exponents: A's row maxima over the four quarters through shared
            // memory, B's column maxima by warp shuffles
            bool tiny_q = false;
            if constexpr (!preA) {
                if constexpr (FAST) {
                    uint32_t mx = 0, lo = 0;
#pragma unroll
                    for (int p = 0; p < QC; ++p) {
                        const unsigned long long b = (unsigned long long)__double_as_longlong(av[p]);
                        mx = max(mx, (uint32_t)(b >> 32) & 0x7FFFFFFFu);
                        lo |= (uint32_t)b;
                    }
                    s_rkey[q][rloc] = mx | (lo != 0u ? 1u : 0u);
                    // this quarter alone looks like a row of values below 2^-997
                    // (a conservative test: another quarter may hold the row's
                    // large maximum); decided together with the exchange barrier
                    tiny_q = !key_fast(mx | (lo != 0u ? 1u : 0u));
                } else {
                    unsigned long long mx = 0;
#pragma unroll
                    for (int p = 0; p < QC; ++p) {
                        const unsigned long long v = (unsigned long long)__double_as_longlong(av[p]) & 0x7FFFFFFFFFFFFFFFull;
                        mx = v > mx ? v : mx;
                    }
                    s_rmax[q][rloc] = mx;
                }
            }
            if constexpr (!PRE) {
#pragma unroll
                for (int jc = 0; jc < 4; ++jc) {
                    unsigned long long mx = 0;
#pragma unroll
                    for (int h = 0; h < KB; ++h) {
                        const unsigned long long v =
                            (unsigned long long)__double_as_longlong(bv[jc][h]) & 0x7FFFFFFFFFFFFFFFull;
                        mx = v > mx ? v : mx;
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const unsigned long long w = __shfl_xor_sync(0xffffffffu, mx, o);
                        mx = w > mx ? w : mx;
                    }
                    if (lane == 0) s_F[slot][4 * warp + jc] = mx ? exp_of_bits(mx) : 0;
                }
            }
            // row / column exponents exchanged; FAST: any quarter of tiny values
            // anywhere (CTA-uniform) sends this chunk down the exact 64-bit path
            bool slow = !FAST;
            if constexpr (FAST) {
                slow = __syncthreads_or(tiny_q) != 0;
            } else {
                if (!(preA && PRE)) __syncthreads();
            }
            int E = 0, ksh = 0;
            if constexpr (!preA) {
                if constexpr (FAST) {
                    const uint32_t key = max(max(s_rkey[0][rloc], s_rkey[1][rloc]), max(s_rkey[2][rloc], s_rkey[3][rloc]));
                    if (!slow) {
                        E = key_exponent(key);
                        ksh = key_shift(key);
                    } else {
                        unsigned long long mx = 0;
#pragma unroll
                        for (int p = 0; p < QC; ++p) {
                            const unsigned long long v = (unsigned long long)__double_as_longlong(av[p]) & 0x7FFFFFFFFFFFFFFFull;
                            mx = v > mx ? v : mx;
                        }
                        s_rmax[q][rloc] = mx;
                        __syncthreads();
                    }
                }
                if (slow) {
                    unsigned long long mx = s_rmax[0][rloc];
#pragma unroll
                    for (int qq = 1; qq < 4; ++qq) mx = s_rmax[qq][rloc] > mx ? s_rmax[qq][rloc] : mx;
                    E = mx ? exp_of_bits(mx) : 0;
                }
                if (q == 0) s_E[slot][rloc] = E;
            }
            // (3) digits into the planes of this stage (free: their MMAs were
            // waited for when the previous chunk was recombined)
            if constexpr (!preA) {
                uint8_t* dst = planeA + (rloc >> 3) * C_::sbo + (rloc & 7) * 16 + (q * QC / 8) * 128;
                if (!slow) {
                    if constexpr (FAST) {
#pragma unroll
                        for (int g = 0; g < QC / 8; ++g) {
                            uint32_t packed[3][4];
#pragma unroll
                            for (int p = 0; p < 8; p += 2) {
                                float2 f1, f2, f3;
                                digits_bf16_s3_x2(av[8 * g + p], av[8 * g + p + 1], ksh, f1, f2, f3);
                                packed[0][p >> 1] = __byte_perm(__float_as_uint(f1.x), __float_as_uint(f1.y), 0x7632);
                                packed[1][p >> 1] = __byte_perm(__float_as_uint(f2.x), __float_as_uint(f2.y), 0x7632);
                                packed[2][p >> 1] = __byte_perm(__float_as_uint(f3.x), __float_as_uint(f3.y), 0x7632);
                            }
#pragma unroll
                            for (int s2 = 0; s2 < 3; ++s2)
                                *reinterpret_cast<uint4*>(dst + s2 * C_::planeA + g * 128) =
                                    make_uint4(packed[s2][0], packed[s2][1], packed[s2][2], packed[s2][3]);
                        }
                    }
                } else {
#pragma unroll
                    for (int g = 0; g < QC / 8; ++g) {
                        uint32_t packed[S][4];
#pragma unroll
                        for (int p = 0; p < 8; p += 2) {
                            int d0[S], d1[S];
                            make_digits<S, BETA>(av[8 * g + p], E, d0);
                            make_digits<S, BETA>(av[8 * g + p + 1], E, d1);
#pragma unroll
                            for (int s2 = 0; s2 < S; ++s2)
                                packed[s2][p >> 1] =
                                    (uint32_t)digit_bits<FP16>(d0[s2]) | ((uint32_t)digit_bits<FP16>(d1[s2]) << 16);
                        }
#pragma unroll
                        for (int s2 = 0; s2 < S; ++s2)
                            *reinterpret_cast<uint4*>(dst + s2 * C_::planeA + g * 128) =
                                make_uint4(packed[s2][0], packed[s2][1], packed[s2][2], packed[s2][3]);
                    }
                }
            }
            // This chunk's units and the tile records.  Mode 2's first chunk of
            // a tile (after the CTA's first) need not wait for the newest cp.async
            // group, the record just issued at the tile's start (needed two
            // tiles later): its units came one iteration earlier, by cp.async
            // or, with BULK, by bulk copies on the stage's unit barrier.  A unit
            // wait that expires stops the CTA after the barrier below, before
            // any tensor-core work reads the stage.
            if (MODE == 2 && (BULK || (c == 0 && iter > 0)))
                asm volatile("cp.async.wait_group 1;\n" ::: "memory");
            else
                asm volatile("cp.async.wait_group 0;\n" ::: "memory");
            if constexpr (BULK) {
                if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&s_ubar[stage]), (ucount[stage] - 1u) & 1u)))
                    s_fail[(iter - 1) & 1] = 1;
            }
            if constexpr (!PRE) {
#pragma unroll
                for (int jc = 0; jc < 4; ++jc) {
                    const int j = 4 * warp + jc;
                    const int F = s_F[slot][j];
                    uint8_t* dst = planeB + (j >> 3) * C_::sbo + (j & 7) * 16;
#pragma unroll
                    for (int h = 0; h < KB; ++h) {
                        const int kk = lane + 32 * h;
                        int dg[S];
                        make_digits<S, BETA>(bv[jc][h], F, dg);
#pragma unroll
                        for (int s2 = 0; s2 < S; ++s2)
                            *reinterpret_cast<uint16_t*>(dst + s2 * C_::planeB + (kk >> 3) * 128 + (kk & 7) * 2) =
                                digit_bits<FP16>(dg[s2]);
                    }
                }
            }
            // (3b) PRELOAD: the next chunk's A into registers (this chunk's
            // digits are in shared memory), so the loads run during steps 4 and 5
            if constexpr (PRELOAD) {
                if (c + 1 < nch) {
                    load_chunk(d, m0, n0, k0 + KC);
                } else if (tn < n_items) {
                    load_chunk(nxt.d, nxt.row0, nxt.col0, 0);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncthreads();
            if (s_fail[(iter - 1) & 1]) {   // the previous chunk's recombination failed somewhere
                failed = true;
                break;
            }
            // (4) one thread issues the chunk's tensor-core work
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                bool first_of_acc[NACC];
#pragma unroll
                for (int g = 0; g < NACC; ++g) first_of_acc[g] = true;
#pragma unroll
                for (int s1 = 1; s1 <= S; ++s1) {
#pragma unroll
                    for (int t1 = 1; t1 <= S; ++t1) {
                        if (s1 + t1 > S + 1) continue;
                        const int g = acc_of<FP16, S>(s1, t1);
                        const uint32_t dcol = tmem + (uint32_t)(stage * NACC * kTN + g * kTN);
                        const uint32_t a_base = smem_u32(planeA + (s1 - 1) * C_::planeA);
                        const uint32_t b_base = smem_u32(planeB + (t1 - 1) * C_::planeB);
#pragma unroll
                        for (int kq = 0; kq < KC / 16; ++kq) {
                            const uint64_t ad = make_desc(a_base + kq * 256, C_::sbo);
                            const uint64_t bd = make_desc(b_base + kq * 256, C_::sbo);
                            const uint32_t accum = first_of_acc[g] ? 0u : 1u;
                            first_of_acc[g] = false;
                            asm volatile(
                                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dcol),
                                "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
                        }
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                                 smem_u32(&s_bar[stage]))
                             : "memory");
            }
            last_commit = iter;
            const uint32_t parity_prev = (uint32_t)(((iter - 1) >> 1) & 1);
            bool prev_done = true;
            // (5) MODE 2: the next chunk's units into the other stage as soon as
            // the previous chunk's tensor-core work (which read its planes) is
            // done, so the copy runs during the recombination (the recombination's
            // own wait on the same phase then returns at once)
            if constexpr (MODE == 2) {
                if (have_prev)
                    prev_done = __all_sync(0xffffffffu, mbar_wait(smem_u32(&s_bar[prev.stage]), parity_prev));
                if (prev_done) {
                    if (c + 1 < nch) {
                        copy_units(entry, m0, n0, nch, c + 1, stage ^ 1, slot_next);
                    } else if (tn < n_items) {
                        copy_units(nxt.entry, nxt.row0, nxt.col0, (nxt.d.k + KC - 1) / KC, 0, stage ^ 1, slot_next);
                    }
                }
            }
            // (6) recombine the previous chunk while this one runs
            if (have_prev) {
                const bool ok = prev_done && recombine(parity_prev);
                if (!ok) s_fail[iter & 1] = 1;   // the CTA stops after the next barrier
                if (prev.last) {
                    if (ok) store_prev();
                    load_c0(d, m0, n0);   // chunk c is chunk 0 of this tile; consumed next iteration
                }
            }
            prev.C = d.C;
            prev.m = d.m;
            prev.n = d.n;
            prev.ldc = d.ldc;
            prev.row0 = m0;
            prev.col0 = n0;
            prev.c = c;
            prev.stage = stage;
            prev.slot = slot;
            prev.last = (c == nch - 1);
            have_prev = true;
        }
        if (failed) break;
        t = tn;
        ++ti;
    }
    __syncthreads();
    if (s_fail[0] | s_fail[1]) failed = true;   // set in the last iteration
    if (have_prev && !failed) {
        const bool ok = recombine((uint32_t)(((iter - 1) >> 1) & 1));
        if (__syncthreads_or(!ok)) failed = true;
        if (!failed) store_prev();
    }
    if (failed) {
        // a wait expired: give the tensor-core work in flight one more bounded
        // wait before the TMEM it writes is released, and report the failure
        if (last_commit >= 0)
            mbar_wait(smem_u32(&s_bar[last_commit & 1]), (uint32_t)((last_commit >> 1) & 1));
        if (tid == 0) atomicExch(status, 1);
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");   // no copy may land after the CTA exits
    if constexpr (BULK) {   // nor a bulk copy: the last fill of each stage (bounded)
        for (int sg = 0; sg < 2; ++sg)
            if (ucount[sg] > 0u) mbar_wait(smem_u32(&s_ubar[sg]), (ucount[sg] - 1u) & 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
}

template <bool FP16, int S, int MODE>
cudaError_t launch_mode(const STile* items, int n_items, int* status, float* dump,
                        int test_stall, const uint8_t* bunits, const long long* bfirst, const uint8_t* aunits,
                        const long long* afirst, cudaStream_t s) {
    const int smem = Cfg<FP16, S>::smem;
    cudaError_t e = cudaFuncSetAttribute(k_split<FP16, S, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (n_items <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::max(1, std::min(n_items, sms));
    k_split<FP16, S, MODE><<<grid, kThreadsS, smem, s>>>(items, n_items, status, dump, test_stall, bunits,
                                                         bfirst, aunits, afirst);
    return cudaGetLastError();
}

// Items [0, n_b) take mode 1 (or 0 without pre-sliced B), items [n_b, n_items)
// mode 2 (their entries have pre-sliced A): two launches in stream order.
template <bool FP16, int S>
cudaError_t launch_t(const STile* items, int n_items, int n_b, int* status, float* dump, int test_stall,
                     const uint8_t* bunits, const long long* bfirst, const uint8_t* aunits, const long long* afirst,
                     cudaStream_t s) {
    if (bunits == nullptr)
        return launch_mode<FP16, S, 0>(items, n_items, status, dump, test_stall, nullptr, nullptr, nullptr, nullptr,
                                       s);
    cudaError_t e = launch_mode<FP16, S, 1>(items, n_b, status, dump, test_stall, bunits, bfirst, nullptr, nullptr, s);
    if (e == cudaSuccess && n_items > n_b)
        e = launch_mode<FP16, S, 2>(items + n_b, n_items - n_b, status, dump, test_stall, bunits, bfirst, aunits,
                                    afirst, s);
    return e;
}

template <bool FP16, int S>
cudaError_t slice_t(bool a_side, const DevDesc* descs, const BUnit* units, int n_units, uint8_t* out,
                    cudaStream_t s) {
    if (n_units <= 0) return cudaSuccess;
    if (a_side)
        k_slice_a<FP16, S><<<n_units, kThreadsS, 0, s>>>(descs, units, out);
    else
        k_slice_b<FP16, S><<<n_units, kThreadsS, 0, s>>>(descs, units, out);
    return cudaGetLastError();
}

cudaError_t slice_prec(int precision, bool a_side, const DevDesc* descs, const BUnit* units, int n_units,
                       uint8_t* out, cudaStream_t s) {
    switch (precision) {
        case LRB_PREC_SPLIT_BF16_S3: return slice_t<false, 3>(a_side, descs, units, n_units, out, s);
        case LRB_PREC_SPLIT_BF16_S4: return slice_t<false, 4>(a_side, descs, units, n_units, out, s);
        case LRB_PREC_SPLIT_FP16_S3: return slice_t<true, 3>(a_side, descs, units, n_units, out, s);
        case LRB_PREC_SPLIT_FP16_S4: return slice_t<true, 4>(a_side, descs, units, n_units, out, s);
        default: return cudaErrorInvalidValue;
    }
}

size_t unit_bytes(int precision, bool a_side) {
    switch (precision) {
        case LRB_PREC_SPLIT_BF16_S3: return a_side ? Cfg<false, 3>::unitA : Cfg<false, 3>::unitB;
        case LRB_PREC_SPLIT_BF16_S4: return a_side ? Cfg<false, 4>::unitA : Cfg<false, 4>::unitB;
        case LRB_PREC_SPLIT_FP16_S3: return a_side ? Cfg<true, 3>::unitA : Cfg<true, 3>::unitB;
        default: return a_side ? Cfg<true, 4>::unitA : Cfg<true, 4>::unitB;
    }
}

cudaError_t launch_prec(int precision, const STile* items, int n_items, int n_b, int* status, float* dump,
                        int test_stall, const uint8_t* bunits, const long long* bfirst, const uint8_t* aunits,
                        const long long* afirst, cudaStream_t s) {
    switch (precision) {
        case LRB_PREC_SPLIT_BF16_S3:
            return launch_t<false, 3>(items, n_items, n_b, status, dump, test_stall, bunits, bfirst, aunits, afirst, s);
        case LRB_PREC_SPLIT_BF16_S4:
            return launch_t<false, 4>(items, n_items, n_b, status, dump, test_stall, bunits, bfirst, aunits, afirst, s);
        case LRB_PREC_SPLIT_FP16_S3:
            return launch_t<true, 3>(items, n_items, n_b, status, dump, test_stall, bunits, bfirst, aunits, afirst, s);
        case LRB_PREC_SPLIT_FP16_S4:
            return launch_t<true, 4>(items, n_items, n_b, status, dump, test_stall, bunits, bfirst, aunits, afirst, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

struct SplitPlan {
    int precision = 0;
    int test_stall = 0;
    void* dmem = nullptr;
    DevDesc* d_descs = nullptr;
    STile* d_items = nullptr;
    int* d_status = nullptr;
    int n_items = 0;
    // pre-sliced B (nullptr: the kernel slices B itself) and A (entries with
    // several column tiles only); one allocation, freed through bunits
    uint8_t* bunits = nullptr;
    BUnit* d_units = nullptr;
    long long* d_bfirst = nullptr;
    int n_units = 0;
    uint8_t* aunits = nullptr;
    BUnit* d_aunits = nullptr;
    long long* d_afirst = nullptr;
    int n_aunits = 0;
    int n_items_b = 0;   // items [0, n_items_b) have A sliced in the kernel, the rest pre-sliced
};

STile make_tile(const lrb_gemm_desc& d, size_t entry, int row0, int col0) {
    STile t;
    std::memcpy(&t.d, &d, sizeof(DevDesc));
    t.entry = (int32_t)entry;
    t.row0 = row0;
    t.col0 = col0;
    t.pad = 0;
    return t;
}

void build_items(const lrb_gemm_desc* descs, size_t count, std::vector<STile>& items) {
    items.clear();
    for (size_t e = 0; e < count; ++e)
        for (int c0 = 0; c0 < descs[e].n; c0 += kTN)
            for (int r0 = 0; r0 < descs[e].m; r0 += kTM) items.push_back(make_tile(descs[e], e, r0, c0));
}

cudaError_t launch_raw(int precision, const STile* d_items, int n_items, int* d_status, cudaStream_t s) {
    return launch_prec(precision, d_items, n_items, n_items, d_status, nullptr, 0, nullptr, nullptr, nullptr, nullptr,
                       s);
}

int chunk_len(int precision) {
    return (precision == LRB_PREC_SPLIT_FP16_S3 || precision == LRB_PREC_SPLIT_FP16_S4) ? 32 : 64;
}
int digit_count(int precision) {
    return (precision == LRB_PREC_SPLIT_BF16_S3 || precision == LRB_PREC_SPLIT_FP16_S3) ? 3 : 4;
}

// Entries whose A digit planes are made by the pre-pass: those with several
// 64-column tiles, whose 128-row A tiles would otherwise be sliced once per
// column tile.  (Pre-slicing A of single-column-tile entries too was measured
// slower: 15.4 vs 14.0 ms on the 2048-entry T-form batch; the planes' extra
// HBM traffic outweighs the integer work it moves out of the main kernel.)
bool pre_a(const lrb_gemm_desc& d) { return d.n > kTN; }

lrb_status create(int device, int sms, const lrb_gemm_desc* descs, size_t count, int precision, SplitPlan** out,
                  lrb_plan_info* info, int test_stall) {
    (void)device;
    (void)sms;
    *out = nullptr;
    // tiles of entries with one column tile first (their A is sliced in the
    // kernel), then the entries whose A is pre-sliced (several column tiles)
    std::vector<STile> items;
    for (int pass = 0; pass < 2; ++pass)
        for (size_t e = 0; e < count; ++e)
            if (pre_a(descs[e]) == (pass == 1))
                for (int c0 = 0; c0 < descs[e].n; c0 += kTN)
                    for (int r0 = 0; r0 < descs[e].m; r0 += kTM) items.push_back(make_tile(descs[e], e, r0, c0));
    size_t n_items_b = 0;
    for (size_t e = 0; e < count; ++e)
        if (!pre_a(descs[e])) n_items_b += (size_t)((descs[e].n + kTN - 1) / kTN) * ((descs[e].m + kTM - 1) / kTM);
    if (items.size() > 0x7fffffffull) {
        set_last_error("too many split-precision tiles");
        return LRB_ERR_INVALID;
    }
    SplitPlan* p = new SplitPlan();
    p->precision = precision;
    p->test_stall = test_stall;
    const size_t o_items = ((sizeof(DevDesc) * count + 255) / 256) * 256;
    const size_t o_status = o_items + ((sizeof(STile) * std::max<size_t>(items.size(), 1) + 255) / 256) * 256;
    cudaError_t ce = cudaMalloc(&p->dmem, o_status + 256);
    if (ce != cudaSuccess) {
        delete p;
        set_last_error("split plan device memory");
        return LRB_ERR_NOMEM;
    }
    p->d_descs = (DevDesc*)p->dmem;
    p->d_items = (STile*)((char*)p->dmem + o_items);
    p->d_status = (int*)((char*)p->dmem + o_status);
    p->n_items = (int)items.size();
    p->n_items_b = (int)n_items_b;
    ce = cudaMemcpy(p->d_descs, descs, sizeof(DevDesc) * count, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess && !items.empty())
        ce = cudaMemcpy(p->d_items, items.data(), sizeof(STile) * items.size(), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemset(p->d_status, 0, 256);
    if (ce != cudaSuccess) {
        cudaFree(p->dmem);
        delete p;
        set_last_error("split plan upload");
        return LRB_ERR_DEVICE;
    }
    // B units: every (entry, 64-column tile, k-chunk); A units: every (entry,
    // 128-row tile, k-chunk) of entries with more than one column tile.
    // Sliced by pre-passes when they fit in memory (else the kernel slices).
    {
        const int kc = chunk_len(precision);
        std::vector<BUnit> bu, au;
        std::vector<long long> bfirst(count), afirst(count, -1);
        for (size_t e = 0; e < count; ++e) {
            bfirst[e] = (long long)bu.size();
            for (int c0 = 0; c0 < descs[e].n; c0 += kTN)
                for (int k0 = 0; k0 < descs[e].k; k0 += kc) bu.push_back(BUnit{(int32_t)e, c0, k0, 0});
            if (pre_a(descs[e])) {
                afirst[e] = (long long)au.size();
                for (int r0 = 0; r0 < descs[e].m; r0 += kTM)
                    for (int k0 = 0; k0 < descs[e].k; k0 += kc) au.push_back(BUnit{(int32_t)e, r0, k0, 0});
            }
        }
        auto up = [](size_t x) { return (x + 255) / 256 * 256; };
        const size_t ubB = unit_bytes(precision, false), ubA = unit_bytes(precision, true);
        const size_t oB = 0, oBu = oB + up(ubB * bu.size()), oBf = oBu + up(sizeof(BUnit) * bu.size());
        const size_t oA = oBf + up(sizeof(long long) * count), oAu = oA + up(ubA * au.size());
        const size_t oAf = oAu + up(sizeof(BUnit) * au.size()), total = oAf + up(sizeof(long long) * count);
        void* mem = nullptr;
        if (bu.size() < 0x7fffffffull && au.size() < 0x7fffffffull && cudaMalloc(&mem, total) == cudaSuccess) {
            char* b = (char*)mem;
            p->bunits = (uint8_t*)(b + oB);
            p->d_units = (BUnit*)(b + oBu);
            p->d_bfirst = (long long*)(b + oBf);
            p->n_units = (int)bu.size();
            if (!au.empty()) {
                p->aunits = (uint8_t*)(b + oA);
                p->d_aunits = (BUnit*)(b + oAu);
                p->d_afirst = (long long*)(b + oAf);
                p->n_aunits = (int)au.size();
            }
            ce = cudaMemcpy(p->d_units, bu.data(), sizeof(BUnit) * bu.size(), cudaMemcpyHostToDevice);
            if (ce == cudaSuccess)
                ce = cudaMemcpy(p->d_bfirst, bfirst.data(), sizeof(long long) * count, cudaMemcpyHostToDevice);
            if (ce == cudaSuccess && !au.empty())
                ce = cudaMemcpy(p->d_aunits, au.data(), sizeof(BUnit) * au.size(), cudaMemcpyHostToDevice);
            if (ce == cudaSuccess && !au.empty())
                ce = cudaMemcpy(p->d_afirst, afirst.data(), sizeof(long long) * count, cudaMemcpyHostToDevice);
            if (ce != cudaSuccess) {
                cudaFree(mem);
                cudaFree(p->dmem);
                delete p;
                set_last_error("split plan upload");
                return LRB_ERR_DEVICE;
            }
        } else {
            cudaGetLastError();   // a failed allocation leaves the in-kernel slicing
        }
    }
    info->items = p->n_items;
    info->groups = 1;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    info->grid = std::max(1, std::min(p->n_items, nsm));
    *out = p;
    return LRB_OK;
}

// The pre-passes, then the main kernel.
cudaError_t launch_with(SplitPlan* p, float* dump, cudaStream_t s) {
    if (p->bunits) {
        cudaError_t e = slice_prec(p->precision, false, p->d_descs, p->d_units, p->n_units, p->bunits, s);
        if (e == cudaSuccess && p->aunits)
            e = slice_prec(p->precision, true, p->d_descs, p->d_aunits, p->n_aunits, p->aunits, s);
        if (e != cudaSuccess) return e;
    }
    return launch_prec(p->precision, p->d_items, p->n_items, p->bunits ? p->n_items_b : p->n_items,
                       p->d_status, dump, p->test_stall, p->bunits, p->d_bfirst, p->aunits, p->d_afirst, s);
}

cudaError_t launch(SplitPlan* p, cudaStream_t s) { return launch_with(p, nullptr, s); }

cudaError_t launch_dump(SplitPlan* p, float* dump, cudaStream_t s) { return launch_with(p, dump, s); }

int read_status(SplitPlan* p, cudaStream_t s, int* value) {
    cudaError_t e = cudaMemcpyAsync(value, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? 0 : -1;
}

void destroy(SplitPlan* p) {
    if (!p) return;
    if (p->bunits) cudaFree(p->bunits);
    if (p->dmem) cudaFree(p->dmem);
    delete p;
}

}  // namespace split
}  // namespace lrb
