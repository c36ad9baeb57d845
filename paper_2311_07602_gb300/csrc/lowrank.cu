// Producers and consumers of low-rank blocks A ~= U diag(S) V (Eq. 1, Sec. 2),
// batched over independent blocks like the low-rank product itself.
//
//  * randomized SVD (the producer Sec. 2 cites: Halko, Martinsson and Tropp):
//    Y = A Omega, Q = orth(Y), q power iterations Q~ = orth(A^T Q),
//    Q = orth(A Q~); then A^T Q = Q2 R2, R2^T = U~ Sigma W^T, U = Q U~_r,
//    S = Sigma_r, V = W_r^T Q2^T (the SVD of B = Q^T A = R2^T Q2^T);
//  * expansion D += (U diag(S)) V;
//  * rounded addition (whose first step Sec. 2 says is the low-rank product):
//    [U1 S1, U2 S2] = Q1 R1, [V1; V2]^T = Q2 R2, R1 R2^T = U~ Sigma W^T,
//    U = Q1 U~_r, S = Sigma_r, V = W_r^T Q2^T.
//
// Every product with a block-sized operand goes through the persistent FP64
// GEMM kernel (transposed and overwriting forms), which is bound by the FP64
// pipe.  The new kernels are the tall-skinny orthonormalisation (Householder
// QR, one CTA per matrix, the explicit Q formed in place) and the small
// l x l SVD (one-sided Jacobi, one CTA per matrix, in shared memory); both
// are a few percent of the flops of the products with A.  The whole sequence
// of a plan is captured once as a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lowrank.h"

namespace lrb {
namespace lowrank {
namespace {

// ---------------------------------------------------------------- kernels

struct QrDesc {            // Y (rows x cols, ldy) -> explicit Q in place; R (cols x cols, ldr) if non-null
    double* Y;
    double* R;
    int32_t rows, cols, ldy, ldr;
};

struct SvdDesc {           // M = X Y^T (X == nullptr: M = Y^T), l x l, ld l
    const double* X;
    const double* Y;
    double* Ut;            // l x l: left singular vectors, columns in descending order of sigma
    double* W;             // l x l: right singular vectors, same order
    double* sig;           // l singular values, descending
    double* S;             // the caller's r leading values
    int32_t l, r;
};

struct PackDesc {          // dst = [src1 diag(s1), src2 diag(s2)] or its transposed-rows form
    const double* src1;
    const double* s1;
    const double* src2;
    const double* s2;
    double* dst;
    int32_t rows, c1, c2, ld1, ld2, ldd;
};

constexpr int kQrThreads = 512;
constexpr int kQrWarps = kQrThreads / 32;
constexpr int kSvdMaxThreads = 512;
constexpr int kMaxSweeps = 40;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
// Every thread receives the block's sum.  The threads' partials go to shared
// memory and warp 0 alone adds them (16 per lane, then a butterfly), so the
// sum costs ~21 warp-wide FP64 adds instead of 5 per warp: on this GPU a
// warp-wide FP64 add costs the FP64 pipe the same for any number of active
// lanes.  red holds kQrThreads + 1 doubles; the result is red[kQrThreads].
__device__ double block_sum(double v, double* red) {
    __syncthreads();                 // the previous result has been read
    red[threadIdx.x] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < kQrWarps; ++k) t += red[threadIdx.x + 32 * k];
        t = warp_sum(t);
        if (threadIdx.x == 0) red[kQrThreads] = t;
    }
    __syncthreads();
    return red[kQrThreads];
}
__device__ double block_max(double v, double* red) {
    __syncthreads();
    red[threadIdx.x] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < kQrWarps; ++k) t = fmax(t, red[threadIdx.x + 32 * k]);
        t = warp_max(t);
        if (threadIdx.x == 0) red[kQrThreads] = t;
    }
    __syncthreads();
    return red[kQrThreads];
}

// One warp applies H = I - tau v v^T to rows [j, m) of column y:
// y <- y - tau (v^T y) v.  Trip counts are the same for every lane (a lane
// past the end is predicated off in the last step only), and four
// independent partial sums keep a column's loads in flight together.
__device__ __forceinline__ void reflect_column(const double* __restrict__ v, double* y, int j, int m, double tau,
                                               int lane) {
    double d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;
    int base = j;
    for (; base + 128 <= m; base += 128) {
        const int i = base + lane;
        d0 = fma(v[i], y[i], d0);
        d1 = fma(v[i + 32], y[i + 32], d1);
        d2 = fma(v[i + 64], y[i + 64], d2);
        d3 = fma(v[i + 96], y[i + 96], d3);
    }
    const int tail = base;
    for (; base < m; base += 32) {
        const int i = base + lane;
        if (i < m) d0 = fma(v[i], y[i], d0);
    }
    const double t = tau * warp_sum((d0 + d1) + (d2 + d3));
    for (base = j; base + 128 <= m; base += 128) {
        const int i = base + lane;
        y[i] = fma(-t, v[i], y[i]);
        y[i + 32] = fma(-t, v[i + 32], y[i + 32]);
        y[i + 64] = fma(-t, v[i + 64], y[i + 64]);
        y[i + 96] = fma(-t, v[i + 96], y[i + 96]);
    }
    for (base = tail; base < m; base += 32) {
        const int i = base + lane;
        if (i < m) y[i] = fma(-t, v[i], y[i]);
    }
}

// Householder QR of one tall matrix per CTA (rows >= cols), the reflectors
// H_j = I - tau_j v_j v_j^T with v_j(j) = 1 chosen so H_j x = beta e_j,
// beta = -sign(x_j) ||x|| (Golub and Van Loan, Sec. 5.1), applied column by
// column (a warp per trailing column).  Then R is copied out and
// Q = H_0 ... H_{cols-1} [I; 0] is formed in place, backwards.  A zero column
// gives tau = 0 (H = I), so rank-deficient input still yields an orthonormal
// Q.  The matrix is worked on in place in global memory (the panels of the
// resident CTAs stay in L2), the current reflector in shared memory; three
// CTAs per SM (40 registers) fill each other's barrier and scalar phases.
// (Staging a whole panel in shared memory leaves room for one CTA per SM and
// measured slower.)
__global__ void __launch_bounds__(kQrThreads, 3) k_house_qr(const QrDesc* __restrict__ descs) {
    extern __shared__ __align__(16) double sm[];
    __shared__ double red[kQrThreads + 1];
    __shared__ double s_tau[LRB_LR_MAX_L];
    __shared__ double s_par[3];
    const QrDesc d = descs[blockIdx.x];
    const int m = d.rows, l = d.cols;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double* v = sm;
    double* P = d.Y;
    const size_t ld = (size_t)d.ldy;

    for (int j = 0; j < l; ++j) {
        double* x = P + (size_t)j * ld;
        double ssq = 0.0;
        for (int i = j + 1 + tid; i < m; i += kQrThreads) ssq = fma(x[i], x[i], ssq);
        ssq = block_sum(ssq, red);
        int e2 = 0;                           // ||x(j+1:m)|| = 2^e2 sqrt(ssq)
        if (!(ssq >= 0x1p-968 && ssq <= 0x1p968)) {
            // possible under- or overflow: again, scaled by a power of two near the largest entry
            double mx = 0.0;
            for (int i = j + 1 + tid; i < m; i += kQrThreads) mx = fmax(mx, fabs(x[i]));
            mx = block_max(mx, red);
            ssq = 0.0;
            if (mx > 0.0) {
                frexp(mx, &e2);
                const double isc = ldexp(1.0, -e2);
                double s2 = 0.0;
                for (int i = j + 1 + tid; i < m; i += kQrThreads) {
                    const double t = x[i] * isc;
                    s2 = fma(t, t, s2);
                }
                ssq = block_sum(s2, red);
            }
        }
        // the reflector's scalars, by warp 0 alone (a warp-wide FP64 operation
        // costs the pipe the same for one lane as for 32): s_par = {tau, beta, scal}
        if (warp == 0) {
            const double alpha = x[j];
            const double xnorm = ldexp(sqrt(ssq), e2);
            double tau = 0.0, beta = alpha, scal = 0.0;
            if (xnorm > 0.0) {
                beta = -copysign(hypot(alpha, xnorm), alpha);
                tau = (beta - alpha) / beta;
                scal = 1.0 / (alpha - beta);
            }
            if (lane == 0) {
                s_par[0] = tau;
                s_par[1] = beta;
                s_par[2] = scal;
                s_tau[j] = tau;
                v[j] = 1.0;
            }
        }
        __syncthreads();
        const double tau = s_par[0], scal = s_par[2];
        for (int i = j + 1 + tid; i < m; i += kQrThreads) {
            const double t = x[i] * scal;
            x[i] = t;
            v[i] = t;
        }
        __syncthreads();   // v complete
        if (tid == 0) x[j] = s_par[1];
        if (tau != 0.0)
            for (int c = j + 1 + warp; c < l; c += kQrWarps) reflect_column(v, P + (size_t)c * ld, j, m, tau, lane);
        __syncthreads();
    }
    if (d.R != nullptr) {
        for (int e = tid; e < l * l; e += kQrThreads) {
            const int i = e % l, c = e / l;
            d.R[(size_t)i + (size_t)c * (size_t)d.ldr] = i <= c ? P[(size_t)i + (size_t)c * ld] : 0.0;
        }
    }
    __syncthreads();
    for (int j = l - 1; j >= 0; --j) {
        double* x = P + (size_t)j * ld;
        const double tau = s_tau[j];
        for (int i = j + 1 + tid; i < m; i += kQrThreads) v[i] = x[i];
        if (tid == 0) v[j] = 1.0;
        __syncthreads();
        if (tau != 0.0)
            for (int c = j + 1 + warp; c < l; c += kQrWarps) reflect_column(v, P + (size_t)c * ld, j, m, tau, lane);
        for (int i = tid; i < m; i += kQrThreads) x[i] = i < j ? 0.0 : (i == j ? 1.0 - tau : -tau * v[i]);
        __syncthreads();
    }
}

// Column pair k of round `round` in the round-robin order of L players
// (player L-1 fixed, the others rotate); a pair with q >= l is a bye.
__device__ __forceinline__ void jacobi_pair(int round, int k, int L, int& p, int& q) {
    p = k == 0 ? round : (round + k) % (L - 1);
    q = k == 0 ? L - 1 : (round - k + (L - 1)) % (L - 1);
    if (p > q) {
        const int t = p;
        p = q;
        q = t;
    }
}

// Lanes per column pair in k_jacobi_svd: the power of two T <= 32, with
// pairs x T <= limit threads and at least two warps, that minimises the FP64
// instructions of a round.  A warp instruction holds the FP64 pipe for the
// same time whatever the number of active lanes, so a round costs each
// working warp 11 ceil(l / T) instructions (3 dot-product FMAs and 8
// rotation operations per row a lane owns), 3 log2 T (the butterfly sums)
// and about 12 (the rotation angle).  Batches put several cores on every SM,
// so the total over the warps counts (one warp issuing back to back keeps a
// sub-partition's FP64 pipe busy), not the busiest sub-partition; at least
// two warps spread a core over two sub-partitions.  For l = 26..32 that is
// T = 4, two warps per core (T = 8 with four took a rounded addition of 512
// pairs, 32 x 32 cores, from 7.76 to 8.06 ms).
__host__ __device__ inline int jacobi_lanes(int l, int limit) {
    const int np = ((l + 1) & ~1) / 2;
    int best = 1, best_cost = 0x7fffffff;
    for (int T = 1, lg = 0; T <= 32 && np * T <= limit; T *= 2, ++lg) {
        const int warps = (np * T + 31) / 32;
        const int cost = warps < 2 ? 0x3fffffff : warps * (11 * ((l + T - 1) / T) + 3 * lg + 12);
        if (cost < best_cost) {
            best_cost = cost;
            best = T;
        }
    }
    return best;
}

// Threads of a k_jacobi_svd launch whose matrices have l <= maxl.
int jacobi_threads(int maxl) {
    int t = 32;
    for (int l = 2; l <= maxl; ++l) {
        const int np = ((l + 1) & ~1) / 2;
        t = std::max(t, (np * jacobi_lanes(l, kSvdMaxThreads) + 31) / 32 * 32);
    }
    return t;
}

// SVD of the small matrix M = X Y^T, one CTA per matrix, everything in
// shared memory (leading dimension lm = l | 1: odd, so that lanes on one row
// of different columns hit different banks).
//
// Preconditioning (Drmac and Veselic, "New fast and accurate Jacobi SVD
// algorithm", 2008): a Householder QR with column pivoting (Businger and
// Golub), M P = Q R, and the one-sided Jacobi method then runs on R^T, whose
// columns are much closer to orthogonal; cores of rounded additions, sums of
// two graded spectra, need about a third fewer rotations that way.  Column j
// of the QR takes the remaining column of largest norm (smallest index on
// ties); one thread owns each column (lanes = columns), so a reflector's dot
// products and updates cost one warp instruction per row for 32 columns.
//
// One-sided Jacobi (Hestenes) on X = R^T: a sweep visits every column pair
// once in round-robin order (l/2 disjoint pairs per round).  A group of T
// lanes (jacobi_lanes) owns one pair of a round: each lane sums the three dot
// products over its rows, a butterfly gives every lane of the group the same
// sums (the same two partials are added at each step, in either order),
// every lane derives the same rotation, and each lane rotates its rows of X
// and of the accumulated rotations V.  Pairs of a round touch disjoint
// columns, so a round needs one barrier.  A pair is rotated when
// |x_p . x_q| > tol ||x_p|| ||x_q||.  At convergence X V = U_x Sigma with
// orthogonal columns, so M = (Q V) Sigma (P U_x)^T: sigma_c = ||X(:, c)||,
// the left singular vectors are Q V (Q applied to V by its reflectors), the
// right ones P U_x with U_x(:, c) = X(:, c) / sigma_c (zero when sigma_c =
// 0); both are written in descending order of sigma.  A sweep limit bounds
// the iteration; hitting it sets the status word and writes the last iterate.
__global__ void __launch_bounds__(kSvdMaxThreads) k_jacobi_svd(const SvdDesc* __restrict__ descs,
                                                              int* __restrict__ status) {
    extern __shared__ __align__(16) double sm[];
    __shared__ int s_rot[2];
    const SvdDesc d = descs[blockIdx.x];
    const int l = d.l, lm = l | 1;
    double* M = sm;                 // M, then R, then X = R^T; l x l, ld lm
    double* V = M + l * lm;         // accumulated rotations
    double* H = V + l * lm;         // reflectors below the diagonal (v_j(j) = 1 implied)
    double* sg = H + l * lm;        // squared trailing column norms, later sigma
    double* tau = sg + l;
    int* perm = reinterpret_cast<int*>(tau + l);
    int* piv = perm + l;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;

    for (int e = tid; e < l * l; e += nt) {
        const int i = e % l, c = e / l;
        double s;
        if (d.X != nullptr) {
            s = 0.0;
            for (int p = 0; p < l; ++p) s = fma(d.X[i + p * l], d.Y[c + p * l], s);
        } else {
            s = d.Y[c + i * l];
        }
        M[i + c * lm] = s;
        V[i + c * lm] = i == c ? 1.0 : 0.0;
    }
    // Column c of the QR belongs to lane c % 32 of warp (w0 + c / 32) % nw; w0
    // varies with the CTA so that the CTAs on one SM spread this serial work
    // over the SM's sub-partitions.
    const int w0 = (int)(blockIdx.x % (unsigned)nw);
    const int cown = lane + 32 * ((warp - w0 + nw) % nw);
    __syncthreads();
    if (cown < l) {
        double s = 0.0;
        for (int i = 0; i < l; ++i) s = fma(M[i + cown * lm], M[i + cown * lm], s);
        sg[cown] = s;
        piv[cown] = cown;
    }
    __syncthreads();
    for (int j = 0; j < l; ++j) {
        if (warp == w0) {
            // pivot: the largest remaining norm (non-negative doubles order like their bit patterns)
            long long best = -1;
            int bi = j;
            for (int c = j + lane; c < l; c += 32) {
                const long long v = __double_as_longlong(sg[c]);
                if (v > best) {
                    best = v;
                    bi = c;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) {
                    best = ob;
                    bi = oi;
                }
            }
            if (bi != j) {
                for (int i = lane; i < l; i += 32) {
                    const double t = M[i + j * lm];
                    M[i + j * lm] = M[i + bi * lm];
                    M[i + bi * lm] = t;
                }
                if (lane == 0) {
                    const double t = sg[j];
                    sg[j] = sg[bi];
                    sg[bi] = t;
                    const int p = piv[j];
                    piv[j] = piv[bi];
                    piv[bi] = p;
                }
            }
            __syncwarp();
            // reflector of column j: H_j = I - tau v v^T maps M(j:l, j) to beta e_j
            const double alpha = M[j + j * lm];
            double s2 = 0.0;
            for (int i = j + 1 + lane; i < l; i += 32) s2 = fma(M[i + j * lm], M[i + j * lm], s2);
            s2 = warp_sum(s2);
            double t = 0.0, scal = 0.0, beta = alpha;
            if (s2 > 0.0) {
                beta = -copysign(hypot(alpha, sqrt(s2)), alpha);
                t = (beta - alpha) / beta;
                scal = 1.0 / (alpha - beta);
            }
            for (int i = j + 1 + lane; i < l; i += 32) {
                H[i + j * lm] = M[i + j * lm] * scal;
                M[i + j * lm] = 0.0;
            }
            if (lane == 0) {
                M[j + j * lm] = beta;
                tau[j] = t;
            }
        }
        __syncthreads();
        if (cown > j && cown < l) {
            double* x = M + cown * lm;
            const double* v = H + j * lm;
            double w = x[j];
            for (int i = j + 1; i < l; ++i) w = fma(v[i], x[i], w);
            const double tw = tau[j] * w;
            x[j] -= tw;
            double s = 0.0;
            for (int i = j + 1; i < l; ++i) {
                const double y = fma(-tw, v[i], x[i]);
                x[i] = y;
                s = fma(y, y, s);
            }
            sg[cown] = s;
        }
        __syncthreads();
    }
    // X = R^T, in place
    for (int e = tid; e < l * l; e += nt) {
        const int i = e % l, c = e / l;
        if (i < c) {
            const double t = M[i + c * lm];
            M[i + c * lm] = M[c + i * lm];
            M[c + i * lm] = t;
        }
    }
    __syncthreads();

    const double tol = (double)l * 2.220446049250313e-16;   // l x 2^-52
    const int L = (l + 1) & ~1;                              // players, with a bye for odd l
    const int NP = L / 2;                                    // pairs per round
    const int T = jacobi_lanes(l, nt);
    const int k = tid / T, g = tid % T;                      // pair group, lane within it
    bool converged = false;
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
        const int cur = sweep & 1;
        if (tid == 0) s_rot[cur] = 0;
        __syncthreads();
        for (int round = 0; round < L - 1; ++round) {
            int p = 0, q = l;
            if (k < NP) jacobi_pair(round, k, L, p, q);
            double a = 0.0, b = 0.0, gm = 0.0;
            if (q < l) {
                for (int i = g; i < l; i += T) {
                    const double mp = M[i + p * lm], mq = M[i + q * lm];
                    a = fma(mp, mp, a);
                    b = fma(mq, mq, b);
                    gm = fma(mp, mq, gm);
                }
            }
            for (int o = T >> 1; o > 0; o >>= 1) {   // every lane of the warp takes part
                a += __shfl_xor_sync(0xffffffffu, a, o);
                b += __shfl_xor_sync(0xffffffffu, b, o);
                gm += __shfl_xor_sync(0xffffffffu, gm, o);
            }
            // rotate when |g| > tol sqrt(a b), tested as g^2 > tol^2 a b (no square roots)
            if (q < l && gm != 0.0 && gm * gm > a * (tol * tol * b)) {
                // t = tan(theta) of the rotation that makes the pair orthogonal,
                // t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), zeta = (b - a) / 2g.
                // The angle is taken in binary32 (the FP64 divisions and square
                // roots cost more of the FP64 pipe than the whole rotation); c and
                // s then come from t in binary64, c = 1/sqrt(1 + t^2), s = c t, so
                // the rotation is orthogonal to binary64 precision and an inexact
                // angle only leaves a residual that the next sweep removes.
                const float gf = (float)gm, df = (float)(b - a);
                const float zf = df / (2.0f * gf);
                double t;
                if (fabsf(gf) >= 1e-30f && fabsf(gf) <= 1e30f && fabsf(df) <= 1e30f && fabsf(zf) < 1e18f) {
                    const float az = fabsf(zf);
                    t = copysign((double)(1.0f / (az + sqrtf(fmaf(az, az, 1.0f)))), (double)zf);
                } else {                        // zeta or its parts outside binary32's range: binary64
                    const double zeta = (b - a) / (2.0 * gm);
                    const double az = fabs(zeta);
                    const double root = az < 1e100 ? sqrt(fma(az, az, 1.0)) : az;
                    t = copysign(1.0 / (az + root), zeta);
                }
                const double c = rsqrt(fma(t, t, 1.0));
                const double s = c * t;
                if (s != 0.0) {
                    for (int i = g; i < l; i += T) {
                        const double mp = M[i + p * lm], mq = M[i + q * lm];
                        M[i + p * lm] = c * mp - s * mq;
                        M[i + q * lm] = s * mp + c * mq;
                        const double wp = V[i + p * lm], wq = V[i + q * lm];
                        V[i + p * lm] = c * wp - s * wq;
                        V[i + q * lm] = s * wp + c * wq;
                    }
                    if (g == 0) s_rot[cur] = 1;
                }
            }
            __syncthreads();
        }
        if (s_rot[cur] == 0) {
            converged = true;
            break;
        }
    }
    for (int c = tid; c < l; c += nt) {
        double s = 0.0;
        for (int i = 0; i < l; ++i) s = fma(M[i + c * lm], M[i + c * lm], s);
        sg[c] = sqrt(s);
    }
    // Q V: the reflectors applied to each column of V, the last one first
    if (cown < l) {
        double* x = V + cown * lm;
        for (int j = l - 1; j >= 0; --j) {
            const double tj = tau[j];
            if (tj == 0.0) continue;
            const double* v = H + j * lm;
            double w = x[j];
            for (int i = j + 1; i < l; ++i) w = fma(v[i], x[i], w);
            const double tw = tj * w;
            x[j] -= tw;
            for (int i = j + 1; i < l; ++i) x[i] = fma(-tw, v[i], x[i]);
        }
    }
    __syncthreads();
    for (int c = tid; c < l; c += nt) {
        int rank = 0;
        for (int o = 0; o < l; ++o) rank += (sg[o] > sg[c] || (sg[o] == sg[c] && o < c)) ? 1 : 0;
        perm[rank] = c;
    }
    __syncthreads();
    for (int e = tid; e < l * l; e += nt) {
        const int i = e % l, j = e / l;
        const int c = perm[j];
        const double s = sg[c];
        d.Ut[i + j * l] = V[i + c * lm];
        d.W[piv[i] + j * l] = s > 0.0 ? M[i + c * lm] / s : 0.0;
    }
    for (int j = tid; j < l; j += nt) {
        const double s = sg[perm[j]];
        d.sig[j] = s;
        if (j < d.r) d.S[j] = s;
    }
    if (!converged && tid == 0) atomicOr(status, 1);
}

// dst(:, c) = src1(:, c) s1(c) for c < c1, src2(:, c - c1) s2(c - c1) after
// (a null scale means 1); one CTA per entry.
__global__ void __launch_bounds__(256) k_pack_cols(const PackDesc* __restrict__ descs) {
    const PackDesc d = descs[blockIdx.x];
    const int cols = d.c1 + d.c2;
    for (int c = 0; c < cols; ++c) {
        const bool first = c < d.c1;
        const double* src = first ? d.src1 + (size_t)c * d.ld1 : d.src2 + (size_t)(c - d.c1) * d.ld2;
        const double* sv = first ? d.s1 : d.s2;
        const double sc = sv != nullptr ? sv[first ? c : c - d.c1] : 1.0;
        double* dst = d.dst + (size_t)c * d.ldd;
        for (int i = threadIdx.x; i < d.rows; i += blockDim.x) dst[i] = src[i] * sc;
    }
}

// dst (rows x (c1 + c2), ldd) = [V1; V2]^T for V1 (c1 x rows, ld1) and V2
// (c2 x rows, ld2): 32 x 32 tiles through shared memory, so both the reads
// (along a column of V) and the writes (along a column of dst) are coalesced.
__global__ void __launch_bounds__(256) k_pack_rows_t(const PackDesc* __restrict__ descs) {
    __shared__ double tile[32][33];
    const PackDesc d = descs[blockIdx.x];
    const int cols = d.c1 + d.c2;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int c0 = 0; c0 < cols; c0 += 32) {
        for (int j0 = 0; j0 < d.rows; j0 += 32) {
            for (int jj = ty; jj < 32; jj += 8) {
                const int c = c0 + tx, j = j0 + jj;
                double val = 0.0;
                if (c < cols && j < d.rows)
                    val = c < d.c1 ? d.src1[(size_t)c + (size_t)j * d.ld1]
                                   : d.src2[(size_t)(c - d.c1) + (size_t)j * d.ld2];
                tile[jj][tx] = val;
            }
            __syncthreads();
            for (int cc = ty; cc < 32; cc += 8) {
                const int c = c0 + cc, j = j0 + tx;
                if (c < cols && j < d.rows) d.dst[(size_t)j + (size_t)c * d.ldd] = tile[tx][cc];
            }
            __syncthreads();
        }
    }
}

size_t svd_smem(int l) {
    const size_t lm = (size_t)(l | 1);
    return (3 * lm * l + 2 * (size_t)l) * 8 + 2 * (size_t)l * 4 + 16;
}

// ---------------------------------------------------------------- plans

enum Kind { kRsvd = 1, kExpand = 2, kRoundAdd = 3 };

lrb_status failv(lrb_status s, const char* fmt, size_t e) {
    char buf[200];
    std::snprintf(buf, sizeof buf, fmt, e);
    set_last_error(buf);
    return s;
}

lrb_status fail0(lrb_status s, const char* msg) {
    set_last_error(msg);
    return s;
}

// Byte range of a column-major rows x cols matrix; false on overflow.
struct Rng {
    uint64_t lo, hi;
    bool out;
};
bool range_of(const void* p, int64_t rows, int64_t cols, int64_t ld, bool out, std::vector<Rng>& v) {
    const __int128 last = (__int128)ld * (cols - 1) + rows - 1;
    const __int128 bytes = (last + 1) * 8;
    const __int128 lo = (__int128)(uintptr_t)p;
    if (bytes > ((__int128)1 << 62) || lo + bytes > ((__int128)1 << 64) - 1) return false;
    v.push_back(Rng{(uint64_t)lo, (uint64_t)(lo + bytes), out});
    return true;
}

// Outputs may overlap neither each other nor any input.
bool overlaps(std::vector<Rng>& v) {
    std::vector<Rng> outs;
    for (const Rng& r : v)
        if (r.out) outs.push_back(r);
    std::sort(outs.begin(), outs.end(), [](const Rng& a, const Rng& b) { return a.lo < b.lo; });
    for (size_t i = 1; i < outs.size(); ++i)
        if (outs[i].lo < outs[i - 1].hi) return true;
    for (const Rng& r : v) {
        if (r.out) continue;
        auto it = std::upper_bound(outs.begin(), outs.end(), r.lo, [](uint64_t x, const Rng& o) { return x < o.hi; });
        if (it != outs.end() && it->lo < r.hi) return true;
    }
    return false;
}

bool aligned8(const void* p) { return ((uintptr_t)p & 7u) == 0; }

lrb_status check_block(const lrb_lr_block& b, bool out, size_t e, std::vector<Rng>& rng) {
    if (!b.U || !b.S || !b.V) return failv(LRB_ERR_INVALID, "entry %zu: NULL block pointer", e);
    if (!aligned8(b.U) || !aligned8(b.S) || !aligned8(b.V))
        return failv(LRB_ERR_INVALID, "entry %zu: block pointer not 8-byte aligned", e);
    if (b.m <= 0 || b.n <= 0 || b.r <= 0 || b.ldu < b.m || b.ldv < b.r)
        return failv(LRB_ERR_INVALID, "entry %zu: bad block dimension or leading dimension", e);
    if (b.m > LRB_LR_MAX_ROWS || b.n > LRB_LR_MAX_ROWS)
        return failv(LRB_ERR_UNSUPPORTED, "entry %zu: block rows or columns above LRB_LR_MAX_ROWS", e);
    if (!range_of(b.U, b.m, b.r, b.ldu, out, rng) || !range_of(b.S, b.r, 1, b.r, out, rng) ||
        !range_of(b.V, b.r, b.n, b.ldv, out, rng))
        return failv(LRB_ERR_INVALID, "entry %zu: block extent overflows", e);
    return LRB_OK;
}

}  // namespace

struct LrPlan {
    int kind = 0;
    int device = 0;
    lrb_handle* h = nullptr;
    void* work = nullptr;        // per-entry temporaries
    void* dmem = nullptr;        // device descriptor arrays + status word
    int* d_status = nullptr;
    std::vector<lrb_plan*> gemm;  // sub-plans in launch order of their first use
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

lrb_status cuda_err(cudaError_t e, const char* what) {
    set_last_error((std::string(what) + ": " + cudaGetErrorString(e)).c_str());
    return LRB_ERR_DEVICE;
}

// Sub-plan through the public planner: FP64, tuned tiles, no alias check
// (the temporaries are disjoint by construction; the caller's ranges were
// checked above).
lrb_status sub_plan(LrPlan* p, const std::vector<lrb_gemm_desc>& d, int trans, int overwrite, lrb_plan** out) {
    lrb_plan_opts o = default_plan_opts();
    o.check_alias = 0;
    o.trans = trans;
    o.overwrite = overwrite;
    lrb_status s = lrb_plan_create(p->h, d.data(), d.size(), &o, out);
    if (s == LRB_OK) p->gemm.push_back(*out);
    return s;
}

// Device copies of the kernels' descriptor arrays, one allocation.
struct Uploader {
    std::vector<char> host;
    size_t add(const void* src, size_t bytes) {
        const size_t off = (host.size() + 255) & ~(size_t)255;
        host.resize(off + bytes);
        std::memcpy(host.data() + off, src, bytes);
        return off;
    }
};

template <class T>
const T* at(void* base, size_t off) {
    return reinterpret_cast<const T*>((char*)base + off);
}

// Kernel launches of a plan, recorded as a list so they can be captured.
struct Step {
    enum Op { kGemm, kQr, kSvd, kPack, kPackT } op;
    size_t off;        // descriptor array offset in dmem
    int count;
    size_t smem;
    lrb_plan* g;
    int threads = 0;      // SVD: threads per CTA
};

// A QR step over `count` matrices of at most `rows` rows (the reflector in
// shared memory).
Step qr_step(size_t off, int count, int rows) {
    return Step{Step::kQr, off, count, 8 * (size_t)rows + 16, nullptr};
}

lrb_status set_smem_limits(size_t svd_smem_bytes) {
    cudaError_t e = cudaFuncSetAttribute(k_house_qr, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(8 * LRB_LR_MAX_ROWS + 16));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_jacobi_svd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)svd_smem_bytes);
    return e == cudaSuccess ? LRB_OK : cuda_err(e, "kernel shared-memory limit");
}

// Allocates work/dmem, uploads descriptors, captures the steps into a graph.
lrb_status finish(LrPlan* p, Uploader& up, const std::vector<Step>& steps) {
    const size_t st_off = up.add("\0\0\0\0", 4);
    cudaError_t e = cudaMalloc(&p->dmem, up.host.size());
    if (e != cudaSuccess) return cuda_err(e, "low-rank plan descriptors");
    e = cudaMemcpy(p->dmem, up.host.data(), up.host.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_err(e, "low-rank plan upload");
    p->d_status = (int*)((char*)p->dmem + st_off);
    e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_err(e, "capture stream");
    e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_err(e, "begin capture");
    cudaError_t le = cudaSuccess;
    for (const Step& s : steps) {
        if (le != cudaSuccess) break;
        switch (s.op) {
            case Step::kGemm:
                le = enqueue_fp64_plan(s.g, p->cap);
                break;
            case Step::kQr:
                k_house_qr<<<s.count, kQrThreads, s.smem, p->cap>>>(at<QrDesc>(p->dmem, s.off));
                le = cudaGetLastError();
                break;
            case Step::kSvd:
                k_jacobi_svd<<<s.count, s.threads, s.smem, p->cap>>>(at<SvdDesc>(p->dmem, s.off), p->d_status);
                le = cudaGetLastError();
                break;
            case Step::kPack:
                k_pack_cols<<<s.count, 256, 0, p->cap>>>(at<PackDesc>(p->dmem, s.off));
                le = cudaGetLastError();
                break;
            case Step::kPackT:
                k_pack_rows_t<<<s.count, 256, 0, p->cap>>>(at<PackDesc>(p->dmem, s.off));
                le = cudaGetLastError();
                break;
        }
    }
    e = cudaStreamEndCapture(p->cap, &p->graph);
    if (le != cudaSuccess) return cuda_err(le, "low-rank plan capture");
    if (e != cudaSuccess) return cuda_err(e, "end capture");
    e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    if (e != cudaSuccess) return cuda_err(e, "graph instantiate");
    return LRB_OK;
}

// Work space: a bump allocator over one device allocation (offsets first,
// pointers after the allocation).
struct Bump {
    size_t bytes = 0;
    size_t take(size_t elems) {
        const size_t off = (bytes + 31) & ~(size_t)31;
        bytes = off + elems * 8;
        return off;
    }
};

lrb_status alloc_work(LrPlan* p, size_t bytes) {
    cudaError_t e = cudaMalloc(&p->work, std::max<size_t>(bytes, 256));
    return e == cudaSuccess ? LRB_OK : cuda_err(e, "low-rank plan temporaries");
}

double* wp(LrPlan* p, size_t off) { return (double*)((char*)p->work + off); }

double qr_flops(double rows, double l) { return 2.0 * (2.0 * rows * l * l - 2.0 * l * l * l / 3.0); }

}  // namespace

lrb_status create_rsvd(lrb_handle* h, const lrb_rsvd_desc* d, size_t count, int q, LrPlan** out,
                       lrb_plan_info* info) {
    *out = nullptr;
    if (!d) return fail0(LRB_ERR_INVALID, "host_descs is NULL");
    if (count == 0 || count > 0x7fffffffull) return failv(LRB_ERR_INVALID, "count %zu out of range", count);
    if (q < 0 || q > 8) return fail0(LRB_ERR_INVALID, "power_iters must be 0..8");
    std::vector<Rng> rng;
    double flops = 0, bytes = 0;
    int maxl = 1, maxm = 1, maxn = 1;
    for (size_t e = 0; e < count; ++e) {
        const lrb_rsvd_desc& x = d[e];
        const lrb_lr_block& b = x.out;
        if (!x.A || !x.Omega) return failv(LRB_ERR_INVALID, "entry %zu: NULL A or Omega", e);
        if (!aligned8(x.A) || !aligned8(x.Omega)) return failv(LRB_ERR_INVALID, "entry %zu: pointer not 8-byte aligned", e);
        lrb_status s = check_block(b, true, e, rng);
        if (s != LRB_OK) return s;
        if (x.l < b.r || x.l > std::min(b.m, b.n) || x.lda < b.m || x.ldo < b.n)
            return failv(LRB_ERR_INVALID, "entry %zu: need r <= l <= min(m, n), lda >= m, ldo >= n", e);
        if (x.l > LRB_LR_MAX_L) return failv(LRB_ERR_UNSUPPORTED, "entry %zu: l above LRB_LR_MAX_L", e);
        if (!range_of(x.A, b.m, b.n, x.lda, false, rng) || !range_of(x.Omega, b.n, x.l, x.ldo, false, rng))
            return failv(LRB_ERR_INVALID, "entry %zu: input extent overflows", e);
        const double m = b.m, n = b.n, l = x.l, r = b.r;
        flops += 2.0 * m * n * l * (2 + 2 * q) + (1 + q) * (qr_flops(m, l) + qr_flops(n, l)) + 2.0 * (m + n) * l * r;
        bytes += 8.0 * (m * n + n * l + m * r + r + r * n);
        maxm = std::max(maxm, b.m);
        maxn = std::max(maxn, b.n);
        maxl = std::max(maxl, x.l);
    }
    if (overlaps(rng)) {
        set_last_error("an output range overlaps an input or another output");
        return LRB_ERR_ALIAS;
    }
    LrPlan* p = new LrPlan();
    p->kind = kRsvd;
    p->h = h;
    p->device = handle_info(h).device;
    auto bail = [&](lrb_status s) {
        destroy(p);
        return s;
    };
    lrb_status s = set_smem_limits(svd_smem(maxl));
    if (s != LRB_OK) return bail(s);

    Bump bump;
    struct Off {
        size_t Y, Z, R, Ut, W, sig, Vr;
    };
    std::vector<Off> off(count);
    for (size_t e = 0; e < count; ++e) {
        const size_t m = d[e].out.m, n = d[e].out.n, l = d[e].l, r = d[e].out.r;
        off[e] = Off{bump.take(m * l), bump.take(n * l), bump.take(l * l), bump.take(l * l), bump.take(l * l),
                     bump.take(l), bump.take(n * r)};
    }
    s = alloc_work(p, bump.bytes);
    if (s != LRB_OK) return bail(s);

    std::vector<lrb_gemm_desc> gAO(count), gATY(count), gAZ(count), gU(count), gV(count);
    std::vector<QrDesc> qY(count), qZ(count), qZR(count);
    std::vector<SvdDesc> sv(count);
    std::vector<PackDesc> pt(count);
    for (size_t e = 0; e < count; ++e) {
        const lrb_rsvd_desc& x = d[e];
        const lrb_lr_block& b = x.out;
        double *Y = wp(p, off[e].Y), *Z = wp(p, off[e].Z), *R = wp(p, off[e].R);
        double *Ut = wp(p, off[e].Ut), *W = wp(p, off[e].W), *sig = wp(p, off[e].sig), *Vr = wp(p, off[e].Vr);
        const int m = b.m, n = b.n, l = x.l, r = b.r;
        gAO[e] = lrb_gemm_desc{x.A, x.Omega, Y, m, l, n, x.lda, x.ldo, m};          // Y = A Omega
        gATY[e] = lrb_gemm_desc{x.A, Y, Z, n, l, m, x.lda, m, n};                   // Z = A^T Q
        gAZ[e] = lrb_gemm_desc{x.A, Z, Y, m, l, n, x.lda, n, m};                    // Y = A Q~
        gU[e] = lrb_gemm_desc{Y, Ut, b.U, m, r, l, m, l, b.ldu};                    // U = Q U~_r
        gV[e] = lrb_gemm_desc{Z, W, Vr, n, r, l, n, l, n};                          // V^T = Q2 W_r
        pt[e] = PackDesc{Vr, nullptr, nullptr, nullptr, b.V, r, n, 0, n, 0, b.ldv};  // V = (V^T)^T
        qY[e] = QrDesc{Y, nullptr, m, l, m, 0};
        qZ[e] = QrDesc{Z, nullptr, n, l, n, 0};
        qZR[e] = QrDesc{Z, R, n, l, n, l};
        sv[e] = SvdDesc{nullptr, R, Ut, W, sig, b.S, l, r};
    }
    lrb_plan *pAO, *pATY, *pAZ = nullptr, *pU, *pV;
    if ((s = sub_plan(p, gAO, 0, 1, &pAO)) != LRB_OK || (s = sub_plan(p, gATY, 1, 1, &pATY)) != LRB_OK ||
        (q > 0 && (s = sub_plan(p, gAZ, 0, 1, &pAZ)) != LRB_OK) || (s = sub_plan(p, gU, 0, 1, &pU)) != LRB_OK ||
        (s = sub_plan(p, gV, 0, 1, &pV)) != LRB_OK)
        return bail(s);
    Uploader up;
    const size_t oY = up.add(qY.data(), sizeof(QrDesc) * count);
    const size_t oZ = up.add(qZ.data(), sizeof(QrDesc) * count);
    const size_t oZR = up.add(qZR.data(), sizeof(QrDesc) * count);
    const size_t oS = up.add(sv.data(), sizeof(SvdDesc) * count);
    const size_t oT = up.add(pt.data(), sizeof(PackDesc) * count);
    const int c = (int)count;
    std::vector<Step> steps;
    steps.push_back({Step::kGemm, 0, 0, 0, pAO});
    steps.push_back(qr_step(oY, c, maxm));
    for (int it = 0; it < q; ++it) {
        steps.push_back({Step::kGemm, 0, 0, 0, pATY});
        steps.push_back(qr_step(oZ, c, maxn));
        steps.push_back({Step::kGemm, 0, 0, 0, pAZ});
        steps.push_back(qr_step(oY, c, maxm));
    }
    steps.push_back({Step::kGemm, 0, 0, 0, pATY});
    steps.push_back(qr_step(oZR, c, maxn));
    steps.push_back({Step::kSvd, oS, c, svd_smem(maxl), nullptr, jacobi_threads(maxl)});
    steps.push_back({Step::kGemm, 0, 0, 0, pU});
    steps.push_back({Step::kGemm, 0, 0, 0, pV});
    steps.push_back({Step::kPackT, oT, c, 0, nullptr});
    if ((s = finish(p, up, steps)) != LRB_OK) return bail(s);
    std::memset(info, 0, sizeof(*info));
    info->entries = (int64_t)count;
    info->flops = flops;
    info->alg_bytes = bytes;
    info->precision = LRB_PREC_FP64;
    for (lrb_plan* g : p->gemm) {
        lrb_plan_info gi;
        lrb_plan_get_info(g, &gi);
        info->items += gi.items;
        info->grid = std::max(info->grid, gi.grid);
    }
    info->groups = (int64_t)steps.size();
    *out = p;
    return LRB_OK;
}

lrb_status create_expand(lrb_handle* h, const lrb_expand_desc* d, size_t count, LrPlan** out,
                         lrb_plan_info* info) {
    *out = nullptr;
    if (!d) return fail0(LRB_ERR_INVALID, "host_descs is NULL");
    if (count == 0 || count > 0x7fffffffull) return failv(LRB_ERR_INVALID, "count %zu out of range", count);
    std::vector<Rng> rng;
    double flops = 0, bytes = 0;
    for (size_t e = 0; e < count; ++e) {
        const lrb_expand_desc& x = d[e];
        lrb_status s = check_block(x.blk, false, e, rng);
        if (s != LRB_OK) return s;
        if (!x.D || !aligned8(x.D) || x.ldd < x.blk.m) return failv(LRB_ERR_INVALID, "entry %zu: bad D or ldd", e);
        if (!range_of(x.D, x.blk.m, x.blk.n, x.ldd, true, rng))
            return failv(LRB_ERR_INVALID, "entry %zu: D extent overflows", e);
        const double m = x.blk.m, n = x.blk.n, r = x.blk.r;
        flops += 2.0 * m * n * r + m * r;
        bytes += 8.0 * (m * r + r + r * n + 2 * m * n);
    }
    if (overlaps(rng)) {
        set_last_error("a D range overlaps a block or another D");
        return LRB_ERR_ALIAS;
    }
    LrPlan* p = new LrPlan();
    p->kind = kExpand;
    p->h = h;
    p->device = handle_info(h).device;
    auto bail = [&](lrb_status s) {
        destroy(p);
        return s;
    };
    Bump bump;
    std::vector<size_t> off(count);
    for (size_t e = 0; e < count; ++e) off[e] = bump.take((size_t)d[e].blk.m * d[e].blk.r);
    lrb_status s = alloc_work(p, bump.bytes);
    if (s != LRB_OK) return bail(s);
    std::vector<lrb_gemm_desc> g(count);
    std::vector<PackDesc> pk(count);
    for (size_t e = 0; e < count; ++e) {
        const lrb_lr_block& b = d[e].blk;
        double* Ws = wp(p, off[e]);
        pk[e] = PackDesc{b.U, b.S, nullptr, nullptr, Ws, b.m, b.r, 0, b.ldu, 1, b.m};
        g[e] = lrb_gemm_desc{Ws, b.V, d[e].D, b.m, b.n, b.r, b.m, b.ldv, d[e].ldd};
    }
    lrb_plan* pg;
    if ((s = sub_plan(p, g, 0, 0, &pg)) != LRB_OK) return bail(s);
    Uploader up;
    const size_t oP = up.add(pk.data(), sizeof(PackDesc) * count);
    std::vector<Step> steps{{Step::kPack, oP, (int)count, 0, nullptr}, {Step::kGemm, 0, 0, 0, pg}};
    if ((s = finish(p, up, steps)) != LRB_OK) return bail(s);
    lrb_plan_info gi;
    lrb_plan_get_info(pg, &gi);
    *info = gi;
    info->flops = flops;
    info->alg_bytes = bytes;
    info->groups = (int64_t)steps.size();
    *out = p;
    return LRB_OK;
}

lrb_status create_round_add(lrb_handle* h, const lrb_round_add_desc* d, size_t count, LrPlan** out,
                            lrb_plan_info* info) {
    *out = nullptr;
    if (!d) return fail0(LRB_ERR_INVALID, "host_descs is NULL");
    if (count == 0 || count > 0x7fffffffull) return failv(LRB_ERR_INVALID, "count %zu out of range", count);
    if (count > 0x3fffffffull)   // one QR launch covers 2 x count matrices
        return failv(LRB_ERR_UNSUPPORTED, "count %zu out of range", count);
    std::vector<Rng> rng;
    double flops = 0, bytes = 0;
    int maxl = 1, maxm = 1, maxn = 1;
    for (size_t e = 0; e < count; ++e) {
        const lrb_round_add_desc& x = d[e];
        lrb_status s;
        if ((s = check_block(x.x, false, e, rng)) != LRB_OK || (s = check_block(x.y, false, e, rng)) != LRB_OK ||
            (s = check_block(x.out, true, e, rng)) != LRB_OK)
            return s;
        const int m = x.x.m, n = x.x.n, lc = x.x.r + x.y.r;
        if (x.y.m != m || x.y.n != n || x.out.m != m || x.out.n != n)
            return failv(LRB_ERR_INVALID, "entry %zu: x, y and out must have the same m and n", e);
        if (x.out.r > lc || lc > std::min(m, n))
            return failv(LRB_ERR_INVALID, "entry %zu: need r <= x.r + y.r <= min(m, n)", e);
        if (lc > LRB_LR_MAX_L) return failv(LRB_ERR_UNSUPPORTED, "entry %zu: x.r + y.r above LRB_LR_MAX_L", e);
        const double M = m, N = n, L = lc, r = x.out.r;
        flops += qr_flops(M, L) + qr_flops(N, L) + 2.0 * L * L * L + 2.0 * (M + N) * L * r;
        bytes += 8.0 * ((M + N + 1) * L + (M + N + 1) * r);
        maxm = std::max(maxm, m);
        maxn = std::max(maxn, n);
        maxl = std::max(maxl, lc);
    }
    if (overlaps(rng)) {
        set_last_error("an output range overlaps an input or another output");
        return LRB_ERR_ALIAS;
    }
    LrPlan* p = new LrPlan();
    p->kind = kRoundAdd;
    p->h = h;
    p->device = handle_info(h).device;
    auto bail = [&](lrb_status s) {
        destroy(p);
        return s;
    };
    lrb_status s = set_smem_limits(svd_smem(maxl));
    if (s != LRB_OK) return bail(s);
    Bump bump;
    struct Off {
        size_t Uc, Vt, R1, R2, Ut, W, sig, Vr;
    };
    std::vector<Off> off(count);
    for (size_t e = 0; e < count; ++e) {
        const size_t m = d[e].x.m, n = d[e].x.n, l = d[e].x.r + d[e].y.r, r = d[e].out.r;
        off[e] = Off{bump.take(m * l), bump.take(n * l), bump.take(l * l), bump.take(l * l),
                     bump.take(l * l), bump.take(l * l), bump.take(l),     bump.take(n * r)};
    }
    if ((s = alloc_work(p, bump.bytes)) != LRB_OK) return bail(s);
    std::vector<PackDesc> pu(count), pv(count), pt(count);
    std::vector<QrDesc> q1(count), q2(count);
    std::vector<SvdDesc> sv(count);
    std::vector<lrb_gemm_desc> gU(count), gV(count);
    for (size_t e = 0; e < count; ++e) {
        const lrb_round_add_desc& x = d[e];
        const int m = x.x.m, n = x.x.n, l = x.x.r + x.y.r, r = x.out.r;
        double *Uc = wp(p, off[e].Uc), *Vt = wp(p, off[e].Vt), *R1 = wp(p, off[e].R1), *R2 = wp(p, off[e].R2);
        double *Ut = wp(p, off[e].Ut), *W = wp(p, off[e].W), *sig = wp(p, off[e].sig), *Vr = wp(p, off[e].Vr);
        pu[e] = PackDesc{x.x.U, x.x.S, x.y.U, x.y.S, Uc, m, x.x.r, x.y.r, x.x.ldu, x.y.ldu, m};
        pv[e] = PackDesc{x.x.V, nullptr, x.y.V, nullptr, Vt, n, x.x.r, x.y.r, x.x.ldv, x.y.ldv, n};
        q1[e] = QrDesc{Uc, R1, m, l, m, l};
        q2[e] = QrDesc{Vt, R2, n, l, n, l};
        sv[e] = SvdDesc{R1, R2, Ut, W, sig, x.out.S, l, r};
        gU[e] = lrb_gemm_desc{Uc, Ut, x.out.U, m, r, l, m, l, x.out.ldu};
        gV[e] = lrb_gemm_desc{Vt, W, Vr, n, r, l, n, l, n};                             // V^T = Q2 W_r
        pt[e] = PackDesc{Vr, nullptr, nullptr, nullptr, x.out.V, r, n, 0, n, 0, x.out.ldv};  // V = (V^T)^T
    }
    // The two QRs, and the products for U and V^T, are independent: one
    // launch each over both halves, so neither ends on a half-empty wave.
    q1.insert(q1.end(), q2.begin(), q2.end());
    gU.insert(gU.end(), gV.begin(), gV.end());
    lrb_plan* pUV;
    if ((s = sub_plan(p, gU, 0, 1, &pUV)) != LRB_OK) return bail(s);
    Uploader up;
    const size_t oPU = up.add(pu.data(), sizeof(PackDesc) * count);
    const size_t oPV = up.add(pv.data(), sizeof(PackDesc) * count);
    const size_t oQ = up.add(q1.data(), sizeof(QrDesc) * q1.size());
    const size_t oS = up.add(sv.data(), sizeof(SvdDesc) * count);
    const size_t oT = up.add(pt.data(), sizeof(PackDesc) * count);
    const int c = (int)count;
    std::vector<Step> steps{{Step::kPack, oPU, c, 0, nullptr},
                            {Step::kPackT, oPV, c, 0, nullptr},
                            qr_step(oQ, 2 * c, std::max(maxm, maxn)),
                            {Step::kSvd, oS, c, svd_smem(maxl), nullptr, jacobi_threads(maxl)},
                            {Step::kGemm, 0, 0, 0, pUV},
                            {Step::kPackT, oT, c, 0, nullptr}};
    if ((s = finish(p, up, steps)) != LRB_OK) return bail(s);
    std::memset(info, 0, sizeof(*info));
    info->entries = (int64_t)count;
    info->flops = flops;
    info->alg_bytes = bytes;
    info->precision = LRB_PREC_FP64;
    info->groups = (int64_t)steps.size();
    info->grid = (int)count;
    *out = p;
    return LRB_OK;
}

cudaError_t launch(LrPlan* p, cudaStream_t s) { return cudaGraphLaunch(p->exec, s); }

int read_status(LrPlan* p, cudaStream_t s, int* value) {
    if (cudaStreamSynchronize(s) != cudaSuccess) return 1;
    return cudaMemcpy(value, p->d_status, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess ? 0 : 1;
}

void destroy(LrPlan* p) {
    if (!p) return;
    cudaSetDevice(p->device);
    if (p->cap) cudaStreamSynchronize(p->cap);
    for (lrb_plan* g : p->gemm) lrb_plan_destroy(g);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->cap) cudaStreamDestroy(p->cap);
    if (p->dmem) cudaFree(p->dmem);
    if (p->work) cudaFree(p->work);
    delete p;
}

}  // namespace lowrank
}  // namespace lrb
