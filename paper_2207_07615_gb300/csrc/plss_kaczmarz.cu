// plss_kaczmarz.cu -- identity-sketch PLSS (generalised Kaczmarz), Sec. 7.
//
// For the sketch S_k = [e_{i_1} ... e_{i_k}] the update of eq:pkKacz is
//   p = gamma (a_i - P Theta^{-1} P^T a_i),
//   gamma = r_i / ((||a_i|| - ||d||)(||a_i|| + ||d||)),  d = Theta^{-1/2} P^T a_i,
// with r_i = b_i - a_i^T x, P the stored history and Theta = diag(||p_j||^2).
// The history is kept as the directions q_j = p_j / gamma_j (the projector
// P Theta^{-1} P^T does not depend on the column scale), so every row that
// is not skipped enters the window, even when r_i = 0.
// The window holds at most K updates; once full it is emptied before the
// next row, so every stored update lives on U, the union of the supports of
// the window's rows. P is therefore kept compactly as |U| x K (column j =
// p_j restricted to U) with a column -> slot map, and one row costs
// O(nnz(a_i) K + |U| K) instead of O(n K).
//
// The loop over rows is sequential by nature; for windows of up to 64
// updates one CTA runs one system, and a batch of systems runs as one launch
// with one CTA per system. Larger windows (65..4,096 updates, one system)
// run on the whole GPU (k_kacz_wide below): a row's step is then dominated
// by the product P (Theta^{-1} P^T a_i) over |U| x K entries of the history,
// which one SM cannot stream fast enough. Rows are visited without
// replacement in a fresh permutation per pass (SplitMix64 stream +
// Fisher-Yates shuffle, drawn on the host); ||b - A x|| is tested after
// every pass.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "plss.h"
#include "plss_ctx.h"
#include "plss_dev.cuh"
#include "plss_launch.h"
#include "plss_trace.h"

namespace plss {

constexpr int kKzThreads = 256;
constexpr int kKzWarps = kKzThreads / 32;
constexpr int kKzMaxK = 64;         // one CTA per system up to this window
constexpr int kKwMaxK = 4096;       // whole-GPU window (one system) up to this
constexpr int kKwThreads = 512;
constexpr int kKwWarps = kKwThreads / 32;
constexpr int kKwRowMax = 8192;     // entries of a row held in shared memory

struct KzSys {
    int64_t uoff;       // first U slot of the system (ucols, and rows of P)
    int64_t ucap;       // capacity of U (column stride of P)
    int64_t toff;       // first Theta entry
    int64_t skipped;    // rows skipped (projected norm at rounding level)
    int64_t rows_todo;  // rows to visit in this launch
    int32_t nh, nU;     // updates in the window, columns in U
    int32_t overflow;   // set if U outgrew its capacity (a bounds check)
    int32_t pad;
};

struct KaczState {
    int64_t K = -1;
    int64_t p_entries = 0;
    int32_t *d_slot = nullptr;    // [n_tot] slot of a column in its system's U, or -1
    int32_t *d_ucols = nullptr;   // [sum ucap] global column of each slot
    double *d_P = nullptr;        // per system: column j at P + uoff*K + j*ucap
    double *d_theta = nullptr;    // [nsys*K]
    KzSys *d_sys = nullptr;
    int32_t *d_perm = nullptr;    // [m_tot] local row order of the current pass
    int32_t *h_perm = nullptr;    // pinned
    KzSys *h_sys = nullptr;       // pinned
    std::vector<int64_t> ucap;
    // whole-GPU window (K > kKzMaxK): P is row-major, P[s * K + j]
    bool wide = false;
    int32_t wide_grid = 0;
    int32_t row_max = 0;          // longest row of the system
    double *d_part = nullptr;     // [3 * grid] per-CTA partials (a^T x, ||a||^2, theta)
    double *d_c = nullptr;        // [K] c_j = q_j^T a_i, one owner CTA per j
    uint32_t *d_bar = nullptr;    // grid barrier: [0] arrivals, [1] generation, [2] error
};

struct KzArgs {
    const int32_t *row_ptr;
    const int32_t *col_idx;
    const void *val;
    const SysDesc *desc;
    KzSys *ks;
    const int32_t *perm;
    const double *b;
    double *x;
    int32_t *slot;
    int32_t *ucols;
    double *P;
    double *theta;
    int32_t K;
};

// Fixed-order CTA sum of two doubles (result in thread 0).
__device__ __forceinline__ void kz_sum2(double &a, double &b, double (*sh)[kKzWarps]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    __syncthreads();
    if (lane == 0) {
        sh[0][warp] = a;
        sh[1][warp] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int w = 0; w < kKzWarps; ++w) {
            s0 += sh[0][w];
            s1 += sh[1][w];
        }
        a = s0;
        b = s1;
    }
}

template <typename S>
__global__ void __launch_bounds__(kKzThreads) k_kacz(KzArgs a) {
    __shared__ double sh_c[kKzMaxK];
    __shared__ double sh_red[2][kKzWarps];
    __shared__ double sh_gamma;
    __shared__ int sh_skip;
    __shared__ int sh_store;
    __shared__ int sh_wcnt[kKzWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int sys = blockIdx.x;
    const SysDesc d = a.desc[sys];
    const KzSys ks = a.ks[sys];
    const int K = a.K;
    const int64_t ucap = ks.ucap;
    const S *__restrict__ val = static_cast<const S *>(a.val);
    int32_t *U = a.ucols + ks.uoff;
    double *P = a.P + ks.uoff * int64_t(K);
    double *th = a.theta + ks.toff;
    int nh = ks.nh, nU = ks.nU;
    int64_t skipped = ks.skipped;

    for (int64_t t = 0; t < ks.rows_todo; ++t) {
        const int32_t i = int32_t(d.row_off) + a.perm[d.row_off + t];
        const int32_t s0 = a.row_ptr[i], s1 = a.row_ptr[i + 1];
        if (K > 0 && nh == K) {
            // window full: empty it (and U) before this row
            for (int q = tid; q < nU; q += kKzThreads) a.slot[U[q]] = -1;
            nh = 0;
            nU = 0;
            __syncthreads();
        }
        // c_j = p_j^T a_i for the window, one warp per j
        for (int j = warp; j < nh; j += kKzWarps) {
            double acc = 0.0;
            for (int32_t k = s0 + lane; k < s1; k += 32) {
                const int32_t sl = a.slot[a.col_idx[k]];
                if (sl >= 0) acc = fma(double(val[k]), P[int64_t(j) * ucap + sl], acc);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) sh_c[j] = acc;
        }
        // a_i^T x and ||a_i||^2
        double ax = 0.0, a2 = 0.0;
        for (int32_t k = s0 + tid; k < s1; k += kKzThreads) {
            const double v = double(val[k]);
            ax = fma(v, a.x[a.col_idx[k]], ax);
            a2 = fma(v, v, a2);
        }
        kz_sum2(ax, a2, sh_red);
        if (tid == 0) {
            const double ri = a.b[i] - ax;
            double d2 = 0.0;
            for (int j = 0; j < nh; ++j) d2 += (sh_c[j] * sh_c[j]) / th[j];
            const double na = sqrt(a2), nd = sqrt(d2);
            const double delta = (na - nd) * (na + nd);
            const int skip = !(delta > 1e-14 * a2) ? 1 : 0;
            if (!skip) {
                sh_gamma = ri / delta;
                for (int j = 0; j < nh; ++j) sh_c[j] = sh_c[j] / th[j];
            }
            sh_skip = skip;
        }
        __syncthreads();
        if (sh_skip) {
            ++skipped;
            continue;
        }
        const double gamma = sh_gamma;
        if (K == 0) {
            // classical Kaczmarz: x += gamma a_i on the row's support
            for (int32_t k = s0 + tid; k < s1; k += kKzThreads) {
                const int32_t c = a.col_idx[k];
                a.x[c] = __dadd_rn(a.x[c], __dmul_rn(gamma, double(val[k])));
            }
            __syncthreads();
            continue;
        }
        // new columns of a_i get slots in row order (deterministic)
        const int nU0 = nU;
        for (int32_t base = s0; base < s1; base += kKzThreads) {
            const int32_t k = base + tid;
            const bool in = k < s1;
            const int32_t c = in ? a.col_idx[k] : 0;
            const bool isnew = in && a.slot[c] < 0;
            const unsigned bal = __ballot_sync(0xffffffffu, isnew);
            if (lane == 0) sh_wcnt[warp] = __popc(bal);
            __syncthreads();
            int off = nU, tot = 0;
            for (int w = 0; w < kKzWarps; ++w) {
                if (w < warp) off += sh_wcnt[w];
                tot += sh_wcnt[w];
            }
            if (isnew) {
                const int s = off + __popc(bal & ((1u << lane) - 1u));
                if (s < ucap) {
                    a.slot[c] = s;
                    U[s] = c;
                } else {
                    a.ks[sys].overflow = 1;   // cannot happen: |U| <= K * max row length
                }
            }
            nU += tot;
            __syncthreads();
        }
        // clear the rows of P for new slots and the scratch column nh
        for (int s = nU0 + tid; s < nU; s += kKzThreads)
            for (int j = 0; j < K; ++j) P[int64_t(j) * ucap + s] = 0.0;
        for (int s = tid; s < nU0; s += kKzThreads) P[int64_t(nh) * ucap + s] = 0.0;
        __syncthreads();
        // scatter a_i into column nh
        for (int32_t k = s0 + tid; k < s1; k += kKzThreads)
            P[int64_t(nh) * ucap + a.slot[a.col_idx[k]]] = double(val[k]);
        __syncthreads();
        // q = a_i - sum_j (c_j/theta_j) q_j on U; x += gamma q; theta = ||q||^2.
        // The window keeps the directions q (P Theta^{-1} P^T does not depend
        // on their scale), so a row with r_i = 0 still enters it.
        double tq = 0.0, unused = 0.0;
        for (int s = tid; s < nU; s += kKzThreads) {
            double v = P[int64_t(nh) * ucap + s];
            for (int j = 0; j < nh; ++j) v = __dsub_rn(v, __dmul_rn(sh_c[j], P[int64_t(j) * ucap + s]));
            P[int64_t(nh) * ucap + s] = v;
            const int32_t c = U[s];
            a.x[c] = __dadd_rn(a.x[c], __dmul_rn(gamma, v));
            tq = __dadd_rn(tq, __dmul_rn(v, v));
        }
        kz_sum2(tq, unused, sh_red);
        if (tid == 0) {
            sh_store = tq > 0.0;
            if (tq > 0.0) th[nh] = tq;
        }
        __syncthreads();
        nh += sh_store;
    }
    if (tid == 0) {
        a.ks[sys].nh = nh;
        a.ks[sys].nU = nU;
        a.ks[sys].skipped = skipped;
    }
}

// Classical Kaczmarz (window K = 0): a row step is a dot product, one
// division and a scatter of at most a few dozen entries, so a whole CTA
// spends its time in barriers. Here one warp walks one system: the row's
// entries are spread over the lanes, sums are butterfly shuffles (the same
// fixed order in every lane), and the scatter is made visible to the next
// row by __syncwarp. Everything of the next row that does not depend on x
// (its place in the permutation, offsets, b_i and its first 32 indices and
// values) is loaded while the current row is processed, and the scatter
// reuses the x values the dot product gathered, so a row costs about one
// memory round trip (the gather of x).
template <typename S>
__global__ void __launch_bounds__(kKzThreads) k_kacz0(KzArgs a, int32_t nsys) {
    const int lane = threadIdx.x & 31;
    const int32_t sys = int32_t(blockIdx.x) * kKzWarps + (threadIdx.x >> 5);
    if (sys >= nsys) return;   // whole warp
    const SysDesc d = a.desc[sys];
    const KzSys ks = a.ks[sys];
    const S *__restrict__ val = static_cast<const S *>(a.val);
    const int32_t *perm = a.perm + d.row_off;
    int64_t skipped = ks.skipped;
    // row t: i, [s0, s1), b_i, and the lane's entry of the first 32
    const bool any = ks.rows_todo > 0;
    int32_t i = any ? int32_t(d.row_off) + perm[0] : 0;
    int32_t s0 = any ? a.row_ptr[i] : 0, s1 = any ? a.row_ptr[i + 1] : 0;
    double bi = any ? a.b[i] : 0.0;
    int32_t cq = s0 + lane < s1 ? a.col_idx[s0 + lane] : -1;
    double vq = cq >= 0 ? double(val[s0 + lane]) : 0.0;
    for (int64_t t = 0; t < ks.rows_todo; ++t) {
        const bool more = t + 1 < ks.rows_todo;
        const int32_t in = more ? int32_t(d.row_off) + perm[t + 1] : i;
        const double xq = cq >= 0 ? a.x[cq] : 0.0;
        double ax = fma(vq, xq, 0.0), a2 = fma(vq, vq, 0.0);
        for (int32_t k = s0 + 32 + lane; k < s1; k += 32) {
            const double v = double(val[k]);
            ax = fma(v, a.x[a.col_idx[k]], ax);
            a2 = fma(v, v, a2);
        }
        const int32_t s0n = more ? a.row_ptr[in] : 0, s1n = more ? a.row_ptr[in + 1] : 0;
        const double bin = more ? a.b[in] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ax += __shfl_xor_sync(0xffffffffu, ax, o);
            a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        }
        const double ri = bi - ax;
        const double na = sqrt(a2), nd = sqrt(0.0);
        const double delta = (na - nd) * (na + nd);
        if (!(delta > 1e-14 * a2)) {
            ++skipped;
        } else {
            const double gamma = ri / delta;
            if (cq >= 0) a.x[cq] = __dadd_rn(xq, __dmul_rn(gamma, vq));
            for (int32_t k = s0 + 32 + lane; k < s1; k += 32) {
                const int32_t c = a.col_idx[k];
                a.x[c] = __dadd_rn(a.x[c], __dmul_rn(gamma, double(val[k])));
            }
        }
        __syncwarp();
        i = in;
        s0 = s0n;
        s1 = s1n;
        bi = bin;
        cq = more && s0 + lane < s1 ? a.col_idx[s0 + lane] : -1;
        vq = cq >= 0 ? double(val[s0 + lane]) : 0.0;
    }
    if (lane == 0) a.ks[sys].skipped = skipped;
}

// ---------------------------------------------------------------------------
// Whole-GPU window (K > kKzMaxK, one system)
// ---------------------------------------------------------------------------
//
// Every row takes two phases separated by grid barriers, with the CTAs
// splitting the work and taking the scalar decisions redundantly (each CTA
// sums the same partials in the same order, so every CTA holds the same
// bits):
//   A  c_j = q_j^T a_i for the window's j (each CTA owns a range of j) and
//      partials of a_i^T x and ||a_i||^2 (each CTA owns a range of entries);
//   -- barrier --
//      every CTA: d_j = c_j / theta_j, ||d||^2, delta, r_i, gamma, the skip
//      test, and the slots of the row's new columns (row order);
//   B  q = a_i - P d on U (each CTA owns a range of slots): the new column
//      nh of P, x += gamma q, a partial of theta = ||q||^2;
//   -- barrier --
//      every CTA: theta_nh; nh += 1.
// A full window is emptied before the next row (each CTA clears its slots'
// entries of the column -> slot map, then a barrier). P is row-major over
// the slots, P[s * K + j], so c reads and the product's rows are contiguous.
// The barrier is a counter and a generation word with a time limit: a CTA
// that waits longer than kKwWaitNs sets the error word and returns, and so
// does every other CTA that sees it (the host reports PLSS_ERR_TIMEOUT). The
// launch is cooperative, which guarantees that all CTAs are resident.

constexpr unsigned long long kKwWaitNs = 2000000000ull;   // 2 s per barrier

struct KwArgs {
    const int32_t *row_ptr;
    const int32_t *col_idx;
    const void *val;
    const int32_t *perm;
    const double *b;
    double *x;
    int32_t *slot;     // [n] column -> slot, -1 if not in U
    int32_t *ucols;    // [ucap] slot -> column
    double *P;         // [ucap][K]
    double *theta;     // [K]
    double *c;         // [K]
    double *part;      // [3 * gridDim.x]
    uint32_t *bar;     // arrivals, generation, error
    KzSys *ks;
    int64_t row_off, ucap;
    int32_t K, row_max;
};

__device__ __forceinline__ unsigned long long kw_now() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier with a time limit; returns false (to every thread of the CTA)
// when the error word is set.
__device__ __forceinline__ bool kw_barrier(uint32_t *bar, int *sh_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile uint32_t *vb = bar;
        int ok = vb[2] == 0;
        if (ok) {
            const uint32_t gen = vb[1];
            __threadfence();
            if (atomicAdd(bar, 1u) == gridDim.x - 1) {
                bar[0] = 0;
                __threadfence();
                atomicAdd(bar + 1, 1u);
            } else {
                const unsigned long long t0 = kw_now();
                while (vb[1] == gen) {
                    if (vb[2] != 0) { ok = 0; break; }
                    if (kw_now() - t0 > kKwWaitNs) {
                        atomicExch(bar + 2, 1u);
                        ok = 0;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __threadfence();
        }
        *sh_ok = ok;
    }
    __syncthreads();
    return *sh_ok != 0;
}

// Fixed-order CTA sum of one double (shuffle tree per warp, then the warp
// totals in warp order); the result is returned to every thread.
__device__ __forceinline__ double kw_sum(double v, double *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < kKwWarps; ++w) t += sh[w];
    return t;
}

// Fixed-order CTA sums of N doubles at once (one pair of block barriers);
// the results are returned to every thread.
template <int N>
__device__ __forceinline__ void kw_sums(double (&v)[N], double (*sh)[kKwWarps]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    }
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) sh[i][warp] = v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < N; ++i) {
        double t = 0.0;
        for (int w = 0; w < kKwWarps; ++w) t += sh[i][w];
        v[i] = t;
    }
}

template <typename S>
__global__ void __launch_bounds__(kKwThreads, 1) k_kacz_wide(KwArgs a) {
    extern __shared__ __align__(16) unsigned char kw_smem[];
    const int K = a.K;
    double *s_ith = reinterpret_cast<double *>(kw_smem);         // [K] 1 / theta_j
    double *s_d = s_ith + K;                                       // [K]
    double *s_val = s_d + K;                                       // [row_max]
    int32_t *s_col = reinterpret_cast<int32_t *>(s_val + a.row_max);   // [row_max]
    int32_t *s_slot = s_col + a.row_max;                           // [row_max]
    __shared__ double sh_red[kKwWarps];
    __shared__ double sh_red3[3][kKwWarps];
    __shared__ int32_t sh_cnt[kKwWarps];
    __shared__ double sh_gamma;
    __shared__ int sh_skip, sh_ok;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = int(gridDim.x), bid = int(blockIdx.x);
    const S *__restrict__ val = static_cast<const S *>(a.val);
    KzSys ks = a.ks[0];
    int nh = ks.nh, nU = ks.nU;
    int64_t skipped = ks.skipped;
    for (int j = tid; j < nh; j += kKwThreads) s_ith[j] = 1.0 / a.theta[j];
    // a row's index, bounds and entries do not depend on earlier rows: each
    // row's are loaded during the previous row's second phase (the first
    // row's here), leaving only the slot lookups for after the barrier
    int32_t i = 0;
    int len = 0;
    auto load_row = [&](int64_t t) {
        i = int32_t(a.row_off) + a.perm[a.row_off + t];
        const int32_t s0 = a.row_ptr[i];
        len = a.row_ptr[i + 1] - s0;
        for (int e = tid; e < len; e += kKwThreads) {
            s_col[e] = a.col_idx[s0 + e];
            s_val[e] = double(val[s0 + e]);
        }
    };
    if (ks.rows_todo > 0) load_row(0);
    __syncthreads();

    for (int64_t t = 0; t < ks.rows_todo; ++t) {
        if (nh == K) {
            // window full: empty it before this row
            const int lo = int(int64_t(nU) * bid / G), hi = int(int64_t(nU) * (bid + 1) / G);
            for (int q = lo + tid; q < hi; q += kKwThreads) a.slot[a.ucols[q]] = -1;
            if (!kw_barrier(a.bar, &sh_ok)) return;
            nh = 0;
            nU = 0;
        }
        __syncthreads();   // the row's entries (loaded by every thread) are in place
        for (int e = tid; e < len; e += kKwThreads) s_slot[e] = a.slot[s_col[e]];
        __syncthreads();
        // phase A: c_j (owned j), partials of a^T x and ||a||^2 (owned entries)
        {
            const int jlo = int(int64_t(nh) * bid / G), jhi = int(int64_t(nh) * (bid + 1) / G);
            for (int j = jlo + warp; j < jhi; j += kKwWarps) {
                double acc = 0.0;
                for (int e = lane; e < len; e += 32) {
                    const int32_t sl = s_slot[e];
                    if (sl >= 0) acc = fma(s_val[e], a.P[int64_t(sl) * K + j], acc);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (lane == 0) a.c[j] = acc;
            }
            const int elo = int(int64_t(len) * bid / G), ehi = int(int64_t(len) * (bid + 1) / G);
            double v[2] = {0.0, 0.0};   // a^T x, ||a||^2
            for (int e = elo + tid; e < ehi; e += kKwThreads) {
                v[0] = fma(s_val[e], a.x[s_col[e]], v[0]);
                v[1] = fma(s_val[e], s_val[e], v[1]);
            }
            kw_sums<2>(v, sh_red3);
            if (tid == 0) {
                a.part[bid] = v[0];
                a.part[G + bid] = v[1];
            }
        }
        if (!kw_barrier(a.bar, &sh_ok)) return;
        // the scalars, identically in every CTA
        {
            double v[3] = {0.0, 0.0, 0.0};   // a^T x, ||a||^2, ||d||^2
            for (int q = tid; q < G; q += kKwThreads) {
                v[0] += __ldcg(a.part + q);
                v[1] += __ldcg(a.part + G + q);
            }
            for (int j = tid; j < nh; j += kKwThreads) {
                const double cj = __ldcg(a.c + j);
                const double dj = cj * s_ith[j];
                v[2] = fma(cj, dj, v[2]);
                s_d[j] = dj;
            }
            kw_sums<3>(v, sh_red3);
            const double ax = v[0], a2 = v[1], d2 = v[2];
            if (tid == 0) {
                const double ri = a.b[i] - ax;
                const double na = sqrt(a2), nd = sqrt(d2);
                const double delta = (na - nd) * (na + nd);
                sh_skip = !(delta > 1e-14 * a2) ? 1 : 0;
                sh_gamma = sh_skip ? 0.0 : ri / delta;
            }
            __syncthreads();
        }
        if (sh_skip) {
            ++skipped;
            if (t + 1 < ks.rows_todo) load_row(t + 1);   // this row's entries are no longer read
            // keep c and the partials of this row until every CTA has read them
            if (!kw_barrier(a.bar, &sh_ok)) return;
            continue;
        }
        const double gamma = sh_gamma;
        // slots of the row's new columns, in row order (identical in every CTA)
        const int nU0 = nU;
        for (int base = 0; base < len; base += kKwThreads) {
            const int e = base + tid;
            const bool isnew = e < len && s_slot[e] < 0;
            const unsigned bal = __ballot_sync(0xffffffffu, isnew);
            if (lane == 0) sh_cnt[warp] = __popc(bal);
            __syncthreads();
            int off = nU, tot = 0;
            for (int w = 0; w < kKwWarps; ++w) {
                if (w < warp) off += sh_cnt[w];
                tot += sh_cnt[w];
            }
            if (isnew) s_slot[e] = -2 - (off + __popc(bal & ((1u << lane) - 1u)));   // new: -2 - slot
            nU += tot;
            __syncthreads();
        }
        if (int64_t(nU) > a.ucap) {   // cannot happen: |U| <= min(n, K * row_max)
            if (tid == 0) atomicExch(a.bar + 2, 2u);
            return;
        }
        // phase B on the owned slots [lo, hi)
        const int lo = int(int64_t(nU) * bid / G), hi = int(int64_t(nU) * (bid + 1) / G);
        for (int s = lo + tid; s < hi && s < nU0; s += kKwThreads) a.P[int64_t(s) * K + nh] = 0.0;
        __syncthreads();
        for (int e = tid; e < len; e += kKwThreads) {
            const int32_t code = s_slot[e];
            const int sl = code >= 0 ? code : -2 - code;
            if (sl < lo || sl >= hi) continue;
            if (code < 0) {   // a new slot: its history entries are zero
                a.ucols[sl] = s_col[e];
                a.slot[s_col[e]] = sl;
                for (int j = 0; j < nh; ++j) a.P[int64_t(sl) * K + j] = 0.0;
            }
            a.P[int64_t(sl) * K + nh] = s_val[e];
        }
        __syncthreads();
        double tq = 0.0;
        for (int s = lo + warp; s < hi; s += kKwWarps) {
            const double *row = a.P + int64_t(s) * K;
            double acc = 0.0;
            if (s < nU0)
                for (int j = lane; j < nh; j += 32) acc = fma(row[j], s_d[j], acc);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) {
                const double q = row[nh] - acc;
                a.P[int64_t(s) * K + nh] = q;
                const int32_t c = a.ucols[s];
                a.x[c] = __dadd_rn(a.x[c], __dmul_rn(gamma, q));
                tq = fma(q, q, tq);
            }
        }
        if (t + 1 < ks.rows_todo) load_row(t + 1);   // the scatter above was this row's last use
        tq = kw_sum(tq, sh_red);
        if (tid == 0) a.part[2 * G + bid] = tq;
        if (!kw_barrier(a.bar, &sh_ok)) return;
        double th = 0.0;
        for (int q = tid; q < G; q += kKwThreads) th += __ldcg(a.part + 2 * G + q);
        th = kw_sum(th, sh_red);
        if (th > 0.0) {
            if (tid == 0) {
                s_ith[nh] = 1.0 / th;
                if (bid == 0) a.theta[nh] = th;
            }
            ++nh;
        }
        __syncthreads();
    }
    if (bid == 0 && tid == 0) {
        a.ks[0].nh = nh;
        a.ks[0].nU = nU;
        a.ks[0].skipped = skipped;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

// SplitMix64 (Steele, Lea & Flood 2014): add the golden-ratio increment,
// then mix with two xor-shift-multiply rounds and a final xor-shift.
static inline uint64_t splitmix64(uint64_t &state) {
    state += 0x9e3779b97f4a7c15ULL;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

// Durstenfeld's Fisher-Yates shuffle of 0..m-1, one draw per position from
// the top down, index = draw mod (i + 1).
static void shuffle_rows(uint64_t &state, int32_t *perm, int64_t m) {
    for (int64_t i = 0; i < m; ++i) perm[i] = int32_t(i);
    for (int64_t i = m - 1; i > 0; --i) {
        const int64_t j = int64_t(splitmix64(state) % uint64_t(i + 1));
        std::swap(perm[i], perm[j]);
    }
}

static void kacz_free(KaczState *k) {
    if (!k) return;
    dfree(k->d_slot);
    dfree(k->d_ucols);
    dfree(k->d_P);
    dfree(k->d_theta);
    dfree(k->d_sys);
    dfree(k->d_perm);
    dfree(k->d_part);
    dfree(k->d_c);
    dfree(k->d_bar);
    if (k->h_perm) cudaFreeHost(k->h_perm);
    if (k->h_sys) cudaFreeHost(k->h_sys);
    delete k;
}

void free_extra(plss_ctx *c) {
    kacz_free(c->kacz);
    c->kacz = nullptr;
    free_rhs(c);
    free_general(c);
}

static plss_status kacz_prepare(plss_ctx *c, int64_t K) {
    if (c->kacz && c->kacz->K == K) return PLSS_OK;
    kacz_free(c->kacz);
    c->kacz = nullptr;
    KaczState *k = new KaczState();
    k->K = K;
    std::vector<int32_t> rp(static_cast<size_t>(c->m + 1));
    if (cudaMemcpy(rp.data(), c->d_row_ptr, rp.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
        delete k;
        return fail(PLSS_ERR_CUDA, "reading row_ptr failed");
    }
    int64_t total = 0, row_max = 0;
    k->ucap.resize(size_t(c->nsys));
    for (int32_t s = 0; s < c->nsys; ++s) {
        const SysDesc &d = c->h_desc[size_t(s)];
        int64_t maxlen = 0;
        for (int64_t i = d.row_off; i < d.row_off + d.m; ++i)
            maxlen = std::max<int64_t>(maxlen, rp[size_t(i + 1)] - rp[size_t(i)]);
        row_max = std::max(row_max, maxlen);
        k->ucap[size_t(s)] = K > 0 ? std::max<int64_t>(1, std::min<int64_t>(d.n, K * maxlen)) : 1;
        total += k->ucap[size_t(s)];
    }
    k->wide = K > kKzMaxK;
    k->row_max = int32_t(std::max<int64_t>(row_max, 1));
    if (k->wide) {
        if (c->nsys != 1) {
            delete k;
            return fail(PLSS_ERR_INVALID, "a history window above %d updates needs a single-system context",
                        kKzMaxK);
        }
        if (row_max > kKwRowMax) {
            delete k;
            return fail(PLSS_ERR_INVALID, "a history window above %d updates takes rows of at most %d "
                        "nonzeros (longest row: %lld)", kKzMaxK, kKwRowMax, (long long)row_max);
        }
        k->wide_grid = c->nsm;
    }
    k->p_entries = total * std::max<int64_t>(K, 1);
    plss_status st = PLSS_OK;
    if ((st = dalloc(reinterpret_cast<void **>(&k->d_slot), 4 * size_t(c->n), "slot")) != PLSS_OK ||
        (st = dalloc(reinterpret_cast<void **>(&k->d_ucols), 4 * size_t(total), "U")) != PLSS_OK ||
        (st = dalloc(reinterpret_cast<void **>(&k->d_P), 8 * size_t(k->p_entries), "P")) != PLSS_OK ||
        (st = dalloc(reinterpret_cast<void **>(&k->d_theta), 8 * size_t(c->nsys) * size_t(std::max<int64_t>(K, 1)), "theta")) != PLSS_OK ||
        (st = dalloc(reinterpret_cast<void **>(&k->d_sys), sizeof(KzSys) * size_t(c->nsys), "kz")) != PLSS_OK ||
        (st = dalloc(reinterpret_cast<void **>(&k->d_perm), 4 * size_t(std::max<int64_t>(c->m, 1)), "perm")) != PLSS_OK ||
        (k->wide && (st = dalloc(reinterpret_cast<void **>(&k->d_part), 8 * 3 * size_t(k->wide_grid), "partials")) != PLSS_OK) ||
        (k->wide && (st = dalloc(reinterpret_cast<void **>(&k->d_c), 8 * size_t(K), "c")) != PLSS_OK) ||
        (k->wide && (st = dalloc(reinterpret_cast<void **>(&k->d_bar), 4 * 4, "barrier")) != PLSS_OK)) {
        kacz_free(k);
        return st;
    }
    if (cudaMallocHost(reinterpret_cast<void **>(&k->h_perm), 4 * size_t(std::max<int64_t>(c->m, 1))) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void **>(&k->h_sys), sizeof(KzSys) * size_t(c->nsys)) != cudaSuccess) {
        kacz_free(k);
        return fail(PLSS_ERR_NOMEM, "pinned allocation failed");
    }
    c->kacz = k;
    return PLSS_OK;
}

// Sum over each system's rows of (b - A v)^2 with v in d_x (or zero when
// use_zero), from the per-tile partials of the residual kernel.
static plss_status resid2(plss_ctx *c, cudaStream_t s, bool use_zero, std::vector<double> &out) {
    if (use_zero) {
        cudaError_t e = cudaMemsetAsync(c->d_vin, 0, 8 * size_t(std::max<int64_t>(c->n, 1)), s);
        if (e != cudaSuccess) return fail(PLSS_ERR_CUDA, "memset: %s", cudaGetErrorString(e));
    }
    cudaError_t e = launch_spmv(c->d_row_ptr, c->d_col_idx, c->d_val, c->f32, c->d_rt,
                                int32_t(c->h_rt.size()), use_zero ? c->d_vin : c->d_x, c->d_vout,
                                c->d_b, c->d_part_res, c->grid_r, s);
    if (e != cudaSuccess) return fail(PLSS_ERR_CUDA, "residual kernel: %s", cudaGetErrorString(e));
    std::vector<double> part(c->h_rt.size());
    if (cudaMemcpyAsync(part.data(), c->d_part_res, 8 * part.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(PLSS_ERR_CUDA, "reading residual partials failed");
    out.assign(size_t(c->nsys), 0.0);
    for (int32_t sy = 0; sy < c->nsys; ++sy) {
        const SysDesc &d = c->h_desc[size_t(sy)];
        for (int32_t t = 0; t < d.rt_count; ++t) out[size_t(sy)] += part[size_t(d.rt_begin + t)];
    }
    return PLSS_OK;
}

// One pass of the whole-GPU window: a cooperative launch (all CTAs resident,
// one per SM) after clearing the barrier words.
static plss_status launch_wide(plss_ctx *c, KaczState *kz, cudaStream_t s) {
    KwArgs w;
    w.row_ptr = c->d_row_ptr;
    w.col_idx = c->d_col_idx;
    w.val = c->d_val;
    w.perm = kz->d_perm;
    w.b = c->d_b;
    w.x = c->d_x;
    w.slot = kz->d_slot;
    w.ucols = kz->d_ucols;
    w.P = kz->d_P;
    w.theta = kz->d_theta;
    w.c = kz->d_c;
    w.part = kz->d_part;
    w.bar = kz->d_bar;
    w.ks = kz->d_sys;
    w.row_off = c->h_desc[0].row_off;
    w.ucap = kz->ucap[0];
    w.K = int32_t(kz->K);
    w.row_max = kz->row_max;
    const size_t smem = size_t(2 * kz->K) * 8 + size_t(kz->row_max) * 16;
    void *fn = c->f32 ? reinterpret_cast<void *>(k_kacz_wide<float>) : reinterpret_cast<void *>(k_kacz_wide<double>);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kKwThreads, smem);
    if (e != cudaSuccess || per_sm < 1)
        return fail(PLSS_ERR_CUDA, "identity sketch (wide window): %zu bytes of shared memory per CTA do not fit",
                    smem);
    if (cudaMemsetAsync(kz->d_bar, 0, 4 * 4, s) != cudaSuccess) return fail(PLSS_ERR_CUDA, "memset failed");
    void *args[] = {&w};
    e = cudaLaunchCooperativeKernel(fn, dim3(unsigned(kz->wide_grid)), dim3(kKwThreads), args, smem, s);
    if (e != cudaSuccess) return fail(PLSS_ERR_CUDA, "identity sketch (wide window) launch: %s", cudaGetErrorString(e));
    return PLSS_OK;
}

plss_status run_identity_multi(plss_ctx *c, const double *const *b, const double *const *x0,
                               double *const *xo, const plss_opts *o, plss_result *res) {
    TraceRange tr("plss: solve (identity sketch)");
    plss_status st = check_opts(o);
    if (st != PLSS_OK) return st;
    c->state_valid = false;   // x and b of the context are overwritten: nothing to resume
    if (o->kacz_hist < 0 || o->kacz_hist > kKwMaxK)
        return fail(PLSS_ERR_INVALID, "kacz_hist must be in [0, %d]", kKwMaxK);
    if (o->kacz_hist > kKzMaxK && c->nsys != 1)
        return fail(PLSS_ERR_INVALID, "a history window above %d updates needs a single-system context", kKzMaxK);
    if (o->w_mode != PLSS_W_IDENTITY) return fail(PLSS_ERR_INVALID, "the identity sketch takes W = I");
    cudaStream_t s = static_cast<cudaStream_t>(o->stream);
    const bool dev = o->io_device != 0;
    const int64_t K = o->kacz_hist;
    st = kacz_prepare(c, K);
    if (st != PLSS_OK) return st;
    KaczState *kz = c->kacz;
    for (int32_t sy = 0; sy < c->nsys; ++sy) {
        const SysDesc &d = c->h_desc[size_t(sy)];
        if (d.m > 0 && !b[sy]) return fail(PLSS_ERR_INVALID, "b is NULL (system %d)", sy);
        if ((st = put_vec(c->d_b + d.row_off, b[sy], d.m, dev, s)) != PLSS_OK) return st;
        if ((st = put_vec(c->d_x + d.col_off, x0 ? x0[sy] : nullptr, d.n, dev, s)) != PLSS_OK) return st;
    }
    if (cudaMemsetAsync(kz->d_slot, 0xff, 4 * size_t(std::max<int64_t>(c->n, 1)), s) != cudaSuccess)
        return fail(PLSS_ERR_CUDA, "memset failed");
    std::vector<double> nb2, r2;
    if ((st = resid2(c, s, true, nb2)) != PLSS_OK) return st;
    if ((st = resid2(c, s, false, r2)) != PLSS_OK) return st;
    const int n = c->nsys;
    std::vector<int> active(static_cast<size_t>(n), 0), status(static_cast<size_t>(n), PLSS_NOT_CONVERGED);
    std::vector<int64_t> visited(static_cast<size_t>(n), 0), maxit(static_cast<size_t>(n));
    std::vector<uint64_t> rng(static_cast<size_t>(n));
    std::vector<double> rel(static_cast<size_t>(n), 0.0);
    int64_t uoff = 0;
    for (int32_t sy = 0; sy < n; ++sy) {
        const SysDesc &d = c->h_desc[size_t(sy)];
        KzSys z;
        std::memset(&z, 0, sizeof z);
        z.uoff = uoff;
        z.ucap = kz->ucap[size_t(sy)];
        z.toff = int64_t(sy) * std::max<int64_t>(K, 1);
        uoff += z.ucap;
        kz->h_sys[sy] = z;
        maxit[size_t(sy)] = o->maxit < 0 ? int64_t(d.n) : o->maxit;
        rng[size_t(sy)] = o->seed + uint64_t(sy);
        const double nb = std::sqrt(nb2[size_t(sy)]);
        rel[size_t(sy)] = nb > 0.0 ? std::sqrt(r2[size_t(sy)]) / nb : 0.0;
        if (nb == 0.0 || d.m == 0 || rel[size_t(sy)] <= o->tol) status[size_t(sy)] = PLSS_OK;
        else if (maxit[size_t(sy)] > 0) active[size_t(sy)] = 1;
    }
    KzArgs ka;
    ka.row_ptr = c->d_row_ptr;
    ka.col_idx = c->d_col_idx;
    ka.val = c->d_val;
    ka.desc = c->d_desc;
    ka.ks = kz->d_sys;
    ka.perm = kz->d_perm;
    ka.b = c->d_b;
    ka.x = c->d_x;
    ka.slot = kz->d_slot;
    ka.ucols = kz->d_ucols;
    ka.P = kz->d_P;
    ka.theta = kz->d_theta;
    ka.K = int32_t(K);
    if (cudaEventRecord(c->ev0, s) != cudaSuccess) return fail(PLSS_ERR_CUDA, "event record failed");
    for (;;) {
        bool any = false;
        for (int32_t sy = 0; sy < n; ++sy) {
            const SysDesc &d = c->h_desc[size_t(sy)];
            KzSys &z = kz->h_sys[sy];
            z.rows_todo = 0;
            if (!active[size_t(sy)]) continue;
            z.rows_todo = std::min<int64_t>(d.m, maxit[size_t(sy)] - visited[size_t(sy)]);
            shuffle_rows(rng[size_t(sy)], kz->h_perm + d.row_off, d.m);
            any = true;
        }
        if (!any) break;
        if (cudaMemcpyAsync(kz->d_perm, kz->h_perm, 4 * size_t(c->m), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(kz->d_sys, kz->h_sys, sizeof(KzSys) * size_t(n), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return fail(PLSS_ERR_CUDA, "upload of the row order failed");
        if (kz->wide) {
            if ((st = launch_wide(c, kz, s)) != PLSS_OK) return st;
        } else if (K == 0) {
            const int grid = (n + kKzWarps - 1) / kKzWarps;
            if (c->f32) k_kacz0<float><<<grid, kKzThreads, 0, s>>>(ka, n);
            else k_kacz0<double><<<grid, kKzThreads, 0, s>>>(ka, n);
        } else if (c->f32) {
            k_kacz<float><<<n, kKzThreads, 0, s>>>(ka);
        } else {
            k_kacz<double><<<n, kKzThreads, 0, s>>>(ka);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(PLSS_ERR_CUDA, "kaczmarz kernel: %s", cudaGetErrorString(e));
        if (cudaMemcpyAsync(kz->h_sys, kz->d_sys, sizeof(KzSys) * size_t(n), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return fail(PLSS_ERR_CUDA, "reading the window state failed");
        if (kz->wide) {
            uint32_t bar[3] = {0, 0, 0};
            if (cudaMemcpyAsync(bar, kz->d_bar, sizeof bar, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return fail(PLSS_ERR_CUDA, "reading the barrier state failed");
            if (bar[2] == 1) return fail(PLSS_ERR_TIMEOUT, "identity sketch: a grid barrier waited longer than 2 s");
            if (bar[2] != 0) return fail(PLSS_ERR_CUDA, "identity sketch: support capacity exceeded");
        }
        if ((st = resid2(c, s, false, r2)) != PLSS_OK) return st;
        for (int32_t sy = 0; sy < n; ++sy)
            if (kz->h_sys[sy].overflow) return fail(PLSS_ERR_CUDA, "identity sketch: support capacity exceeded (system %d)", sy);
        for (int32_t sy = 0; sy < n; ++sy) {
            if (!active[size_t(sy)]) continue;
            visited[size_t(sy)] += kz->h_sys[sy].rows_todo;
            const double nb = std::sqrt(nb2[size_t(sy)]);
            rel[size_t(sy)] = std::sqrt(r2[size_t(sy)]) / nb;
            if (rel[size_t(sy)] <= o->tol) {
                status[size_t(sy)] = PLSS_OK;
                active[size_t(sy)] = 0;
            } else if (visited[size_t(sy)] >= maxit[size_t(sy)]) {
                status[size_t(sy)] = PLSS_NOT_CONVERGED;
                active[size_t(sy)] = 0;
            }
        }
    }
    if (cudaEventRecord(c->ev1, s) != cudaSuccess) return fail(PLSS_ERR_CUDA, "event record failed");
    for (int32_t sy = 0; sy < n; ++sy) {
        const SysDesc &d = c->h_desc[size_t(sy)];
        if ((st = get_vec(xo ? xo[sy] : nullptr, c->d_x + d.col_off, d.n, dev, s)) != PLSS_OK) return st;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(PLSS_ERR_CUDA, "synchronize failed");
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    plss_status overall = PLSS_OK;
    for (int32_t sy = 0; sy < n; ++sy) {
        if (res) {
            res[sy].status = status[size_t(sy)];
            res[sy].reserved = 0;
            res[sy].iters = visited[size_t(sy)];
            res[sy].relres_rec = rel[size_t(sy)];
            res[sy].relres_true = rel[size_t(sy)];
            res[sy].seconds = double(ms) * 1e-3;
        }
        if (overall == PLSS_OK && status[size_t(sy)] != PLSS_OK) overall = plss_status(status[size_t(sy)]);
    }
    return overall;
}

plss_status run_identity(plss_ctx *c, const double *b, const double *x0, double *x_out,
                         const plss_opts *o, plss_result *res) {
    const double *bb[1] = {b};
    const double *xx[1] = {x0};
    double *oo[1] = {x_out};
    return run_identity_multi(c, bb, xx, oo, o, res);
}

}  // namespace plss
