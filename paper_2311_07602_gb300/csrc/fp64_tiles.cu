// FP64 tile kernels for batched C_i += A_i * B_i (binary64 throughout, as in
// the paper's experiments, Sec. 7).
//
// On GB300 the FP64 pipe is the bound: about 2 DFMA lanes per clock per SM
// (~1.2 TFLOP/s for the chip), while every other pipe and HBM are 1-2 orders
// of magnitude faster, and a warp's DFMA costs the same whether 1 or 32 lanes
// are active.  So the tile code aims at exactly one issued DFMA per useful
// multiply-add:
//   * C is loaded into the accumulators up front (no separate FP64 add in the
//     epilogue) and stored once, as the paper's fused loop nest writes its
//     result once (Alg. 2, Sec. 4.1);
//   * lanes run along rows, so a ragged tile edge disables whole row slots
//     and whole warps' column groups with warp-uniform branches;
//   * k-steps of 16 are staged in shared memory with cp.async double
//     buffering (operands are read far below HBM speed, so plain 8-byte
//     copies suffice and work for any leading dimension).
// The same tile functions serve the persistent work-queue kernel and the
// one-launch-per-shape kernels, so both give bitwise identical results.
#include <algorithm>
#include <type_traits>

#include "lrb_internal.h"

namespace lrb {

const Variant kVariants[kNumVariants] = {
    // tm, tn, wn, sk, dmma
    {2, 2, 4, 1, 0},    // 0: 64 x 8
    {2, 4, 4, 1, 0},    // 1: 64 x 16
    {2, 8, 4, 1, 0},    // 2: 64 x 32
    {2, 16, 4, 1, 0},   // 3: 64 x 64
    {4, 8, 4, 1, 0},    // 4: 128 x 32
    {4, 16, 4, 1, 0},   // 5: 128 x 64
    {1, 8, 1, 4, 0},    // 6: 32 x 8, k split over 4 warps
    {1, 16, 2, 2, 0},   // 7: 32 x 32, k split over 2 warp pairs
    {0, 4, 0, 0, 1},    // 8: DMMA 64 x 32
    {0, 8, 0, 0, 1},    // 9: DMMA 64 x 64
};

size_t variant_smem_bytes(int v) {
    const Variant& V = kVariants[v];
    size_t stage = 2ull * kBK * (V.bm() + V.bn());
    size_t red = V.dmma ? 0 : (size_t)(V.sk - 1) * V.bm() * V.bn();
    return 8 * (stage > red ? stage : red);
}

size_t max_smem_bytes() {
    size_t m = 0;
    for (int v = 0; v < kNumVariants; ++v) {
        size_t s = variant_smem_bytes(v);
        if (s > m) m = s;
    }
    return m;
}

namespace {

__device__ __forceinline__ void cp_async8(double* smem_dst, const double* src, bool pred) {
    unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    int n = pred ? 8 : 0;   // 0 source bytes: the 8 destination bytes are zero-filled
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Operand forms of a launch (template bits, uniform over the launch):
// kTransA: A is stored k x m and the tile multiplies A^T; kTransB: B is
// stored n x k (B^T); kOverwrite: C = op(A) op(B), the old C is not read.
constexpr int kTransA = 1, kTransB = 2, kOverwrite = 4;

// Stage k-step kt of the tile (rows [m0, m0+BM) of op(A), cols [n0, n0+BN)
// of op(B)) into buffer `buf` as As[kk][ii], Bs[kk][jj]; elements outside the
// entry are zero-filled.  Consecutive threads walk the stored matrix's
// contiguous index, so every form reads whole 128-byte segments.
template <int BM, int BN, int OPS>
__device__ __forceinline__ void stage(const DevDesc& d, int m0, int n0, int h, int wc, int kt,
                                      double* As, double* Bs) {
    const int k0 = kt * kBK;
    const int kmax = min(kBK, d.k - k0);
    if constexpr ((OPS & kTransA) != 0) {
        for (int e = threadIdx.x; e < BM * kBK; e += kThreads) {
            const int kk = e % kBK, ii = e / kBK;
            const bool ok = ii < h && kk < kmax;
            const double* src = ok ? d.A + (size_t)(k0 + kk) + (size_t)(m0 + ii) * (size_t)d.lda : d.A;
            cp_async8(As + kk * BM + ii, src, ok);
        }
    } else {
        for (int e = threadIdx.x; e < BM * kBK; e += kThreads) {
            const int ii = e % BM, kk = e / BM;
            const bool ok = ii < h && kk < kmax;
            const double* src = ok ? d.A + (size_t)(m0 + ii) + (size_t)(k0 + kk) * (size_t)d.lda : d.A;
            cp_async8(As + kk * BM + ii, src, ok);
        }
    }
    if constexpr ((OPS & kTransB) != 0) {
        for (int e = threadIdx.x; e < kBK * BN; e += kThreads) {
            const int jj = e % BN, kk = e / BN;
            const bool ok = kk < kmax && jj < wc;
            const double* src = ok ? d.B + (size_t)(n0 + jj) + (size_t)(k0 + kk) * (size_t)d.ldb : d.B;
            cp_async8(Bs + kk * BN + jj, src, ok);
        }
    } else {
        for (int e = threadIdx.x; e < kBK * BN; e += kThreads) {
            const int kk = e % kBK, jj = e / kBK;
            const bool ok = kk < kmax && jj < wc;
            const double* src = ok ? d.B + (size_t)(k0 + kk) + (size_t)(n0 + jj) * (size_t)d.ldb : d.B;
            cp_async8(Bs + kk * BN + jj, src, ok);
        }
    }
    cp_async_commit();
}

// DFMA tile.  Thread (lane, warp): rows lane + 32 i (i < TM); columns
// wn*TN + j (j < TN) with wn = warp % WN; k-slice wk = warp / WN of every
// k-step.  Accumulators start from C (slice 0) or 0 (other slices); slices
// are added in slice order at the end.
template <int TM, int TN, int WN, int SK, int OPS>
__device__ __forceinline__ void tile_dfma(const DevDesc& d, int m0, int n0, double* smem) {
    constexpr int BM = 32 * TM, BN = WN * TN, KS = kBK / SK;
    static_assert(WN * SK == kThreads / 32, "4 warps");
    double* As = smem;                   // [2][kBK][BM]
    double* Bs = smem + 2 * kBK * BM;    // [2][kBK][BN]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wn = warp % WN, wk = warp / WN;
    const int h = min(BM, d.m - m0);
    const int wc = min(BN, d.n - n0);
    const int ni = (h + 31) >> 5;                       // row slots holding a valid row
    const int nj = max(0, min(TN, wc - wn * TN));       // this warp's valid columns
    const int col0 = n0 + wn * TN;

    double acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;
    if (wk == 0 && (OPS & kOverwrite) == 0) {
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int row = lane + 32 * i;
            if (i < ni && row < h) {
                const double* c = d.C + (size_t)(m0 + row) + (size_t)col0 * (size_t)d.ldc;
#pragma unroll
                for (int j = 0; j < TN; ++j)
                    if (j < nj) acc[i][j] = c[(size_t)j * (size_t)d.ldc];
            }
        }
    }

    const int nk = (d.k + kBK - 1) / kBK;
    stage<BM, BN, OPS>(d, m0, n0, h, wc, 0, As, Bs);
    for (int kt = 0; kt < nk; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < nk) {
            stage<BM, BN, OPS>(d, m0, n0, h, wc, kt + 1, As + (buf ^ 1) * kBK * BM, Bs + (buf ^ 1) * kBK * BN);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const int kmax = min(kBK, d.k - kt * kBK);
        const int kb = wk * KS;
        const int ke = min(kb + KS, kmax);
        const double* as = As + buf * kBK * BM + lane;
        const double* bs = Bs + buf * kBK * BN + wn * TN;
        if (ni == TM && nj == TN) {
#pragma unroll 2
            for (int kk = kb; kk < ke; ++kk) {
                double a[TM], b[TN];
#pragma unroll
                for (int i = 0; i < TM; ++i) a[i] = as[kk * BM + 32 * i];
#pragma unroll
                for (int j = 0; j < TN; ++j) b[j] = bs[kk * BN + j];
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            }
        } else if constexpr (TM * TN <= 16) {
            // Partial tile.  A guard inside one k loop compiles to predicated
            // DFMAs, which occupy the FP64 pipe like executed ones; so each
            // pair of columns gets its own k loop behind a warp-uniform branch
            // (at most one column per warp is wasted), and a tile with fewer
            // valid row slots than TM (here TM <= 2: one slot) runs a loop over
            // that slot alone.  Each accumulator still sums over kk in the
            // same order.  (Tiles with more accumulators keep the single loop
            // below: this form would push them into local memory.)
            auto column_pairs = [&](auto rows_c) {
                constexpr int R = decltype(rows_c)::value;
#pragma unroll
                for (int g = 0; g < TN; g += 2) {
                    if (g < nj) {
                        for (int kk = kb; kk < ke; ++kk) {
                            double a[R];
#pragma unroll
                            for (int i = 0; i < R; ++i) a[i] = as[kk * BM + 32 * i];
                            const double b0 = bs[kk * BN + g];
                            const double b1 = TN > 1 ? bs[kk * BN + g + 1] : 0.0;
#pragma unroll
                            for (int i = 0; i < R; ++i) {
                                acc[i][g] = fma(a[i], b0, acc[i][g]);
                                if (TN > 1) acc[i][g + 1] = fma(a[i], b1, acc[i][g + 1]);
                            }
                        }
                    }
                }
            };
            if constexpr (TM == 1) {
                column_pairs(std::integral_constant<int, 1>());
            } else {
                if (ni == TM)
                    column_pairs(std::integral_constant<int, TM>());
                else
                    column_pairs(std::integral_constant<int, 1>());
            }
        } else {
            for (int kk = kb; kk < ke; ++kk) {
                double a[TM], b[TN];
#pragma unroll
                for (int i = 0; i < TM; ++i) a[i] = as[kk * BM + 32 * i];
#pragma unroll
                for (int j = 0; j < TN; ++j) b[j] = bs[kk * BN + j];
#pragma unroll
                for (int i = 0; i < TM; ++i) {
                    if (i < ni) {
#pragma unroll
                        for (int j = 0; j < TN; ++j)
                            if (j < nj) acc[i][j] = fma(a[i], b[j], acc[i][j]);
                    }
                }
            }
        }
        __syncthreads();
    }

    if constexpr (SK > 1) {
        // k-slices 1..SK-1 hand their partial sums to slice 0 through shared
        // memory (free again after the loop's last barrier).
        double* red = smem;
        const int slot = wn * 32 + lane;
        if (wk > 0) {
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j)
                    red[(((wk - 1) * TM + i) * TN + j) * (32 * WN) + slot] = acc[i][j];
        }
        __syncthreads();
        if (wk == 0) {
#pragma unroll
            for (int q = 1; q < SK; ++q)
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j)
                        acc[i][j] += red[(((q - 1) * TM + i) * TN + j) * (32 * WN) + slot];
        }
        __syncthreads();
    }

    if (wk == 0) {
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int row = lane + 32 * i;
            if (i < ni && row < h) {
                double* c = d.C + (size_t)(m0 + row) + (size_t)col0 * (size_t)d.ldc;
#pragma unroll
                for (int j = 0; j < TN; ++j)
                    if (j < nj) c[(size_t)j * (size_t)d.ldc] = acc[i][j];
            }
        }
    }
}

// FP64 tensor-core tile with mma.sync m8n8k4 (row.col).  Warp w owns rows
// [16 w, 16 w + 16) of a 64 x (8 NF) tile as 2 x NF 8x8 fragments.
// Fragment layout (PTX ISA, f64 m8n8k4): A(8x4): lane holds (lane>>2, lane&3);
// B(4x8): (lane&3, lane>>2); C(8x8): (lane>>2, 2(lane&3) + {0,1}).
template <int NF, int OPS>
__device__ __forceinline__ void tile_dmma(const DevDesc& d, int m0, int n0, double* smem) {
    constexpr int BM = 64, BN = 8 * NF;
    double* As = smem;
    double* Bs = smem + 2 * kBK * BM;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int h = min(BM, d.m - m0);
    const int wc = min(BN, d.n - n0);
    const int r_in = lane >> 2, q4 = lane & 3;

    double acc[2][NF][2];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int nf = 0; nf < NF; ++nf) {
            acc[mi][nf][0] = 0.0;
            acc[mi][nf][1] = 0.0;
            const int row = 16 * warp + 8 * mi + r_in;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int col = 8 * nf + 2 * q4 + q;
                if ((OPS & kOverwrite) == 0 && row < h && col < wc)
                    acc[mi][nf][q] = d.C[(size_t)(m0 + row) + (size_t)(n0 + col) * (size_t)d.ldc];
            }
        }
    const bool mv0 = 16 * warp < h, mv1 = 16 * warp + 8 < h;

    const int nk = (d.k + kBK - 1) / kBK;
    stage<BM, BN, OPS>(d, m0, n0, h, wc, 0, As, Bs);
    for (int kt = 0; kt < nk; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < nk) {
            stage<BM, BN, OPS>(d, m0, n0, h, wc, kt + 1, As + (buf ^ 1) * kBK * BM, Bs + (buf ^ 1) * kBK * BN);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const int kmax = min(kBK, d.k - kt * kBK);
        const double* as = As + buf * kBK * BM;
        const double* bs = Bs + buf * kBK * BN;
        for (int kk0 = 0; kk0 < kmax; kk0 += 4) {       // zero-filled beyond kmax
            const int kk = kk0 + q4;
            double a0 = as[kk * BM + 16 * warp + r_in];
            double a1 = as[kk * BM + 16 * warp + 8 + r_in];
#pragma unroll
            for (int nf = 0; nf < NF; ++nf) {
                if (8 * nf < wc) {
                    double b = bs[kk * BN + 8 * nf + r_in];
                    if (mv0)
                        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                                     : "+d"(acc[0][nf][0]), "+d"(acc[0][nf][1]) : "d"(a0), "d"(b));
                    if (mv1)
                        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                                     : "+d"(acc[1][nf][0]), "+d"(acc[1][nf][1]) : "d"(a1), "d"(b));
                }
            }
        }
        __syncthreads();
    }

#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int nf = 0; nf < NF; ++nf) {
            const int row = 16 * warp + 8 * mi + r_in;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int col = 8 * nf + 2 * q4 + q;
                if (row < h && col < wc)
                    d.C[(size_t)(m0 + row) + (size_t)(n0 + col) * (size_t)d.ldc] = acc[mi][nf][q];
            }
        }
}

// Variant sets of the persistent kernel: SET 0 (slim) holds the tiles that
// fit 102 registers (5 CTAs = 20 warps per SM), SET 1 (narrow) adds the
// 64x64 and 128x32 DFMA tiles (168 registers, 3 CTAs), SET 2 (wide) every
// variant (1 CTA).
template <int SET, int OPS>
__device__ __forceinline__ void run_tile(int variant, const DevDesc& d, int m0, int n0, double* smem) {
    switch (variant) {
        case 0: tile_dfma<2, 2, 4, 1, OPS>(d, m0, n0, smem); break;
        case 1: tile_dfma<2, 4, 4, 1, OPS>(d, m0, n0, smem); break;
        case 2: tile_dfma<2, 8, 4, 1, OPS>(d, m0, n0, smem); break;
        case 3: if constexpr (SET >= 1) tile_dfma<2, 16, 4, 1, OPS>(d, m0, n0, smem); break;
        case 4: if constexpr (SET >= 1) tile_dfma<4, 8, 4, 1, OPS>(d, m0, n0, smem); break;
        case 5: if constexpr (SET >= 2) tile_dfma<4, 16, 4, 1, OPS>(d, m0, n0, smem); break;
        case 6: tile_dfma<1, 8, 1, 4, OPS>(d, m0, n0, smem); break;
        case 7: tile_dfma<1, 16, 2, 2, OPS>(d, m0, n0, smem); break;
        case 8: tile_dmma<4, OPS>(d, m0, n0, smem); break;
        case 9: if constexpr (SET >= 2) tile_dmma<8, OPS>(d, m0, n0, smem); break;
        default: break;   // planner never emits other ids
    }
}

// Persistent kernel: each CTA takes the next tile from the work counter until
// the list (ordered longest-first by the planner) is exhausted.  No CTA ever
// waits for another; the counter is the only shared state.  OPS (operand
// forms, above) is instantiated beyond 0 for the slim set only.
template <int SET, int OPS>
__global__ void __launch_bounds__(kThreads, SET == 0 ? 5 : SET == 1 ? 3 : 1) k_persistent(const DevDesc* __restrict__ descs,
                                                                      const Item* __restrict__ items, int n_items,
                                                                      int* __restrict__ head) {
    extern __shared__ __align__(16) double smem[];
    __shared__ int s_item;
    if (threadIdx.x == 0) s_item = atomicAdd(head, 1);
    __syncthreads();
    int it = s_item;
    while (it < n_items) {
        const Item item = items[it];
        const DevDesc d = descs[item.entry];
        __syncthreads();                                   // every thread has read s_item
        if (threadIdx.x == 0) s_item = atomicAdd(head, 1);  // claim the next tile while this one runs
        run_tile<SET, OPS>(item.variant, d, item.row0, item.col0, smem);
        __syncthreads();
        it = s_item;
    }
}

// One uniform launch for a group of entries sharing (variant, m, n, k):
// block b handles tile (b % tiles) of entry entries[b / tiles].
template <int V>
__global__ void __launch_bounds__(kThreads) k_plain(const DevDesc* __restrict__ descs,
                                                    const int32_t* __restrict__ entries,
                                                    int tiles_m, int tiles_n) {
    extern __shared__ __align__(16) double smem[];
    const int tiles = tiles_m * tiles_n;
    const int t = blockIdx.x % tiles;
    const DevDesc d = descs[entries[blockIdx.x / tiles]];
    const int bm = (V == 8 || V == 9) ? 64 : (V == 4 || V == 5 ? 128 : (V >= 6 ? 32 : 64));
    const int bn = V == 0 ? 8 : V == 1 ? 16 : V == 2 ? 32 : V == 3 ? 64 : V == 4 ? 32 : V == 5 ? 64
                 : V == 6 ? 8 : V == 7 ? 32 : V == 8 ? 32 : 64;
    run_tile<2, 0>(V, d, (t % tiles_m) * bm, (t / tiles_m) * bn, smem);
}

template <int V>
cudaError_t plain_launch(const DevDesc* d_descs, const int32_t* d_entries, int n_entries, int tiles_m,
                         int tiles_n, cudaStream_t s) {
    const size_t smem = variant_smem_bytes(V);
    cudaError_t e = cudaFuncSetAttribute(k_plain<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long blocks = (long long)n_entries * tiles_m * tiles_n;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    k_plain<V><<<(unsigned)blocks, kThreads, smem, s>>>(d_descs, d_entries, tiles_m, tiles_n);
    return cudaGetLastError();
}

}  // namespace

int variant_set(int v) { return (v == 5 || v == 9) ? 2 : (v == 3 || v == 4) ? 1 : 0; }

size_t persistent_smem_bytes(int set) {
    size_t m = 0;
    for (int v = 0; v < kNumVariants; ++v)
        if (variant_set(v) <= set) m = std::max(m, variant_smem_bytes(v));
    return m;
}

namespace {
template <int SET, int OPS>
int blocks_for() {
    int nb = 0;
    const size_t smem = persistent_smem_bytes(SET);
    if (cudaFuncSetAttribute(k_persistent<SET, OPS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_persistent<SET, OPS>, kThreads, smem) != cudaSuccess)
        return 0;
    return nb;
}
}  // namespace

int persistent_blocks_per_sm(int set) {
    if (set >= 2) return blocks_for<2, 0>();
    if (set == 1) return blocks_for<1, 0>();
    // the slim set also serves the transposed / overwriting forms: every
    // instantiation gets its shared-memory attribute here; the launch
    // uses the smallest residency of them
    int nb = blocks_for<0, 0>();
    nb = std::min(nb, blocks_for<0, 1>());
    nb = std::min(nb, blocks_for<0, 2>());
    nb = std::min(nb, blocks_for<0, 3>());
    nb = std::min(nb, blocks_for<0, 4>());
    nb = std::min(nb, blocks_for<0, 5>());
    nb = std::min(nb, blocks_for<0, 6>());
    nb = std::min(nb, blocks_for<0, 7>());
    return nb;
}

cudaError_t launch_persistent(const DevDesc* d_descs, const Item* d_items, int n_items, int* d_head, int grid,
                              cudaStream_t s, int set, int ops) {
    // the shared-memory attribute was set by persistent_blocks_per_sm() when
    // the handle was created (not here: this may run under stream capture)
    if (ops < 0 || ops > 7 || (ops != 0 && set != 0)) return cudaErrorInvalidValue;
    const size_t smem = persistent_smem_bytes(set);
    cudaError_t e = cudaMemsetAsync(d_head, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (n_items <= 0) return cudaSuccess;
    const dim3 g(grid), b(kThreads);
    switch (set <= 0 ? ops : 8 + set) {
        case 0: k_persistent<0, 0><<<g, b, smem, s>>>(d_descs, d_items, n_items, d_head); break;
        case 1: k_persistent<0, 1><<<g, b, smem, s>>>(d_descs, d_items, n_items, d_head); break;
        case 2: k_persistent<0, 2><<<g, b, smem, s>>>(d_descs, d_items, n_items, d_head); break;
        case 3: k_persistent<0, 3><<<g, b, smem, s>>>(d_descs, d_items, n_items, d_head); break;
        case 4: k_persistent<0, 4><<<g, b, smem, s>>>(d_descs, d_items, n_items, d_head); break;
        case 5: k_persistent<0, 5><<<g, b, smem, s>>>(d_descs, d_items, n_items, d_head); break;
        case 6: k_persistent<0, 6><<<g, b, smem, s>>>(d_descs, d_items, n_items, d_head); break;
        case 7: k_persistent<0, 7><<<g, b, smem, s>>>(d_descs, d_items, n_items, d_head); break;
        case 9: k_persistent<1, 0><<<g, b, smem, s>>>(d_descs, d_items, n_items, d_head); break;
        default: k_persistent<2, 0><<<g, b, smem, s>>>(d_descs, d_items, n_items, d_head); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_plain_group(int variant, const DevDesc* d_descs, const int32_t* d_entries, int n_entries,
                               int tiles_m, int tiles_n, cudaStream_t s) {
    switch (variant) {
        case 0: return plain_launch<0>(d_descs, d_entries, n_entries, tiles_m, tiles_n, s);
        case 1: return plain_launch<1>(d_descs, d_entries, n_entries, tiles_m, tiles_n, s);
        case 2: return plain_launch<2>(d_descs, d_entries, n_entries, tiles_m, tiles_n, s);
        case 3: return plain_launch<3>(d_descs, d_entries, n_entries, tiles_m, tiles_n, s);
        case 4: return plain_launch<4>(d_descs, d_entries, n_entries, tiles_m, tiles_n, s);
        case 5: return plain_launch<5>(d_descs, d_entries, n_entries, tiles_m, tiles_n, s);
        case 6: return plain_launch<6>(d_descs, d_entries, n_entries, tiles_m, tiles_n, s);
        case 7: return plain_launch<7>(d_descs, d_entries, n_entries, tiles_m, tiles_n, s);
        case 8: return plain_launch<8>(d_descs, d_entries, n_entries, tiles_m, tiles_n, s);
        case 9: return plain_launch<9>(d_descs, d_entries, n_entries, tiles_m, tiles_n, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lrb
