// Fused low-rank multiplication core, batched: G = A_X (A_{V^T} B_U) B_X
// (Alg. 1; batched over independent blocks as in Alg. 2).  For low-rank
// blocks A = A_U A_X A_{V^T} (rank ra) and B = B_U B_X B_{V^T} (rank rb)
// the product A B is A_U G B_{V^T}; G (ra x rb) is the part whose cost grows
// with the block size k.  The paper fuses the three products into one loop
// nest so the r x r temporaries never go to memory (Alg. 2, Sec. 4.1); here
// one CTA per block keeps C_temp and E_temp in shared memory.
//
// binary64 throughout; the FP64 pipe is the bound on GB300 (arithmetic
// intensity 1-4 flop/byte against a ridge of 0.19), so the kernel issues
// exactly one DFMA per multiply-add of the chain:
//   step 1  C_temp = A_{V^T} B_U: 2x2 register micro-tiles; the threads left
//           over split k, and the k-groups are summed in a fixed order;
//           k is staged with cp.async double buffering;
//   step 2  E_temp = A_X C_temp and step 3 G = E_temp B_X from shared
//           memory (A_X, B_X read through the read-only cache).
// Ranks up to 64 (the paper's sweep uses 8..32).  A plan sizes the kernel for
// its largest rank R: the micro-tile passes per thread (a template argument)
// and the staging area (KL k-rows of both operands per buffer, KL x R
// doubles, with KL larger for small R) -- so that rank-8 and rank-16 plans
// keep several times more CTAs per SM than rank-64 plans, which is what
// hides the load latency of blocks this small.
#include <algorithm>

#include "lrb_internal.h"

namespace lrb {
namespace {

constexpr int kLT = 128;     // threads per CTA
constexpr int kRmax = 64;

__device__ __forceinline__ void cpa8(double* dst, const double* src, bool pred) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(src), "r"(pred ? 8 : 0) : "memory");
}

// stage: doubles per operand and buffer (>= R_plan^2 / 2, so that C_temp and
// E_temp fit in the staging area afterwards); PASSES: 2x2 micro-tiles per
// thread when a block has more than 128 of them.
template <int PASSES>
__global__ void __launch_bounds__(kLT, PASSES <= 2 ? 8 : PASSES == 4 ? 6 : 3) k_lr_chain(const LrDesc* __restrict__ descs,
                                                                                  int stage) {
    extern __shared__ __align__(16) double sm[];
    const LrDesc d = descs[blockIdx.x];
    const int ra = d.ra, rb = d.rb, k = d.k;
    const int tid = threadIdx.x;
    // step-1 staging: [2][KL][R] of A_{V^T} columns and [2][KL][R] of B_U rows,
    // R = max(ra, rb) rounded up to even, KL = stage / R (k-step grows as the
    // rank shrinks, so every k-step carries the same work)
    const int R = ((ra > rb ? ra : rb) + 1) & ~1;
    const int KL = stage / R;
    double* sA = sm;
    double* sB = sm + 2 * stage;
    double* red = sm + 4 * stage;              // [KS][4 P] partial sums
    const int mt = (ra + 1) / 2, nt = (rb + 1) / 2;
    const int P = mt * nt;                      // 2x2 micro-tiles
    const int KS = P >= kLT ? 1 : kLT / P;      // k-groups
    const int passes = (P + kLT - 1) / kLT;     // micro-tiles per thread when P > 128

    auto stage_in = [&](int kt, int buf) {
        const int k0 = kt * KL;
        const int kl = min(KL, k - k0);
        for (int e = tid; e < KL * ra; e += kLT) {
            const int i = e % ra, p = e / ra;
            const bool ok = p < kl;
            cpa8(sA + (buf * KL + p) * R + i, ok ? d.AVT + (size_t)i + (size_t)(k0 + p) * d.ld_avt : d.AVT, ok);
        }
        for (int e = tid; e < KL * rb; e += kLT) {
            const int p = e % KL, j = e / KL;
            const bool ok = p < kl;
            cpa8(sB + (buf * KL + p) * R + j, ok ? d.BU + (size_t)(k0 + p) + (size_t)j * d.ld_bu : d.BU, ok);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    // ---- step 1 ----
    double acc[PASSES][4];
#pragma unroll
    for (int a = 0; a < PASSES; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    const int my_tile = tid % (P < kLT ? P : kLT);
    const int kg = P < kLT ? tid / P : 0;
    const bool active = P >= kLT || tid < P * KS;
    const int nk = (k + KL - 1) / KL;
    // (with KS > 1, KS * P <= 128, so the reduction area holds 4 * 128 doubles)
    stage_in(0, 0);
    for (int kt = 0; kt < nk; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < nk) {
            stage_in(kt + 1, buf ^ 1);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncthreads();
        const int kl = min(KL, k - kt * KL);
        if (active) {
#pragma unroll
            for (int pass = 0; pass < PASSES; ++pass) {
                const int t = my_tile + pass * kLT;
                if (pass >= passes || t >= P) break;
                const int i0 = 2 * (t % mt), j0 = 2 * (t / mt);
                const double* a = sA + buf * KL * R + i0;
                const double* b = sB + buf * KL * R + j0;
                double c00 = acc[pass][0], c10 = acc[pass][1], c01 = acc[pass][2], c11 = acc[pass][3];
                for (int p = kg; p < kl; p += KS) {
                    const double a0 = a[p * R], a1 = a[p * R + 1];
                    const double b0 = b[p * R], b1 = b[p * R + 1];
                    c00 = fma(a0, b0, c00);
                    if (i0 + 1 < ra) c10 = fma(a1, b0, c10);
                    if (j0 + 1 < rb) {
                        c01 = fma(a0, b1, c01);
                        if (i0 + 1 < ra) c11 = fma(a1, b1, c11);
                    }
                }
                acc[pass][0] = c00;
                acc[pass][1] = c10;
                acc[pass][2] = c01;
                acc[pass][3] = c11;
            }
        }
        __syncthreads();
    }
    // k-groups -> C_temp (fixed order), into shared memory (staging is free now)
    double* Ct = sm;                       // ra x rb, column-major, ld ra
    double* Et = sm + 2 * stage;           // ra x rb
    if (KS == 1) {
#pragma unroll
        for (int pass = 0; pass < PASSES; ++pass) {
            const int t = my_tile + pass * kLT;
            if (!active || pass >= passes || t >= P) break;   // (64 < P < 128 leaves threads idle)
            const int i0 = 2 * (t % mt), j0 = 2 * (t / mt);
            Ct[i0 + j0 * ra] = acc[pass][0];
            if (i0 + 1 < ra) Ct[i0 + 1 + j0 * ra] = acc[pass][1];
            if (j0 + 1 < rb) {
                Ct[i0 + (j0 + 1) * ra] = acc[pass][2];
                if (i0 + 1 < ra) Ct[i0 + 1 + (j0 + 1) * ra] = acc[pass][3];
            }
        }
    } else if (active) {
        double* r = red + (size_t)kg * (4 * P) + 4 * my_tile;   // with KS > 1, P < 128: one micro-tile per thread
        r[0] = acc[0][0];
        r[1] = acc[0][1];
        r[2] = acc[0][2];
        r[3] = acc[0][3];
    }
    __syncthreads();
    for (int t = tid; KS > 1 && t < P; t += kLT) {
        double s[4] = {0.0, 0.0, 0.0, 0.0};
        for (int g = 0; g < KS; ++g)
#pragma unroll
            for (int q = 0; q < 4; ++q) s[q] += red[(size_t)g * (4 * P) + 4 * t + q];
        const int i0 = 2 * (t % mt), j0 = 2 * (t / mt);
        Ct[i0 + j0 * ra] = s[0];
        if (i0 + 1 < ra) Ct[i0 + 1 + j0 * ra] = s[1];
        if (j0 + 1 < rb) {
            Ct[i0 + (j0 + 1) * ra] = s[2];
            if (i0 + 1 < ra) Ct[i0 + 1 + (j0 + 1) * ra] = s[3];
        }
    }
    __syncthreads();
    // ---- step 2: E = A_X C_temp ----
    for (int o = tid; o < ra * rb; o += kLT) {
        const int i = o % ra, j = o / ra;
        double e = 0.0;
        for (int q = 0; q < ra; ++q) e = fma(__ldg(d.AX + (size_t)i + (size_t)q * d.ld_ax), Ct[q + j * ra], e);
        Et[o] = e;
    }
    __syncthreads();
    // ---- step 3: G = E B_X ----
    for (int o = tid; o < ra * rb; o += kLT) {
        const int i = o % ra, j = o / ra;
        double g = 0.0;
        for (int q = 0; q < rb; ++q) g = fma(Et[i + q * ra], __ldg(d.BX + (size_t)q + (size_t)j * d.ld_bx), g);
        d.G[(size_t)i + (size_t)j * d.ldg] = g;
    }
}

// Kernel configuration for a plan whose largest rank is rmax: staging KL x R
// with KL = max(32, 768 / R) (R = rmax rounded up to even), passes from the
// micro-tile count.
struct ChainCfg {
    int stage, passes;
};
ChainCfg chain_cfg(int rmax) {
    const int R = std::max(2, (rmax + 1) & ~1);
    const int KL = std::max(32, 768 / R);
    const int P = ((rmax + 1) / 2) * ((rmax + 1) / 2);
    const int pass = (P + kLT - 1) / kLT;
    return ChainCfg{KL * R, pass <= 1 ? 1 : pass <= 2 ? 2 : pass <= 4 ? 4 : 8};
}

template <int PASSES>
cudaError_t launch_chain(const LrDesc* d_descs, int count, int stage, cudaStream_t s) {
    const size_t smem = lr_chain_smem_bytes_for(stage);
    cudaError_t e = cudaFuncSetAttribute(k_lr_chain<PASSES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (count <= 0) return cudaSuccess;
    k_lr_chain<PASSES><<<count, kLT, smem, s>>>(d_descs, stage);
    return cudaGetLastError();
}

}  // namespace

size_t lr_chain_smem_bytes_for(int stage) {
    // staging 4 stage doubles (reused for C_temp and E_temp) + reduction 4 kLT doubles
    return 8 * (size_t)(4 * stage + 4 * kLT + 8);
}

int lr_chain_max_rank() { return kRmax; }

cudaError_t launch_lr_chain(const LrDesc* d_descs, int count, int rmax, cudaStream_t s) {
    const ChainCfg c = chain_cfg(rmax);
    switch (c.passes) {
        case 1: return launch_chain<1>(d_descs, count, c.stage, s);
        case 2: return launch_chain<2>(d_descs, count, c.stage, s);
        case 4: return launch_chain<4>(d_descs, count, c.stage, s);
        default: return launch_chain<8>(d_descs, count, c.stage, s);
    }
}

}  // namespace lrb

