// ccs_device.cuh -- the per-column score and per-row residual, shared by the
// host-driven kernels (ccs_decode.cu) and the persistent engine
// (ccs_engine.cu).
//
// Data read across phases of one persistent launch (r, x_hat, fp, slots,
// slot_cnt, touched, in_slots) is loaded with ld.global.cg (L2, never a
// stale L1 line); the matrix and y are read-only and go through the
// read-only path.
#pragma once

#include "ccs_internal.cuh"

namespace ccs {

// 8-bit fingerprint of a residual entry: 0 exactly when the value is zero
// (+0.0 or -0.0), otherwise a hash of its bits in 1..255.  Equal values have
// equal fingerprints, so a fingerprint count bounds the count of any value.
__device__ __forceinline__ uint8_t fingerprint(double v) {
    const unsigned long long b = value_bits(v);
    if (b == 0ull) return 0;
    unsigned long long h = (b ^ (b >> 31)) * 0x9e3779b97f4a7c15ull;
    const unsigned f = (unsigned)(h >> 56);
    return (uint8_t)(f == 0u ? 1u : f);
}

// Exact score of one column from its d row indices `rows` (stride 1).
// Returns true when the pair (j, omega) is accepted; omega's bits in *omega.
// Equality is equality of binary64 values (bit patterns with -0.0 folded);
// the mode is the most frequent nonzero value, ties to the numerically
// smallest (order_key).  Score: Eq. (15) c_omega - c_0, or Alg. 8 c_omega.
template <int DMAX>
__device__ __forceinline__ bool exact_score(const int32_t *rows, int d, const double *r,
                                            int alpha, int mode,
                                            unsigned long long *omega) {
    unsigned long long v[DMAX];
#pragma unroll
    for (int t = 0; t < DMAX; ++t) v[t] = (t < d) ? value_bits(__ldcg(r + rows[t])) : 0ull;
    int c0 = 0;
#pragma unroll
    for (int t = 0; t < DMAX; ++t) c0 += (t < d) & (v[t] == 0ull);
    int best_cnt = 0;
    unsigned long long best_bits = 0ull, best_key = ~0ull;
#pragma unroll
    for (int a = 0; a < DMAX; ++a) {
        int c = 0;
#pragma unroll
        for (int b = 0; b < DMAX; ++b) c += (b < d) & (v[b] == v[a]);
        const unsigned long long key = order_key(v[a]);
        const bool better = (a < d) && (v[a] != 0ull) &&
                            (c > best_cnt || (c == best_cnt && key < best_key));
        best_cnt = better ? c : best_cnt;
        best_key = better ? key : best_key;
        best_bits = better ? v[a] : best_bits;
    }
    const int score = (mode == CCS_SCORE_COUNT) ? best_cnt : best_cnt - c0;
    *omega = best_bits;
    return best_cnt > 0 && score >= alpha;
}

// Fingerprint bound on the score: with F the largest multiplicity of a
// nonzero fingerprint among the d rows and c0 the number of zero rows,
// every value omega has c_omega <= F, so score <= F - c0 (Eq. (15)) or
// <= F (Alg. 8).  Returns false when no pair of this column can reach alpha.
template <int DMAX>
__device__ __forceinline__ bool may_accept(const uint8_t *fp_smem, const int32_t *rows, int d,
                                           int alpha, int mode) {
    unsigned f[DMAX];
#pragma unroll
    for (int t = 0; t < DMAX; ++t) f[t] = (t < d) ? (unsigned)fp_smem[rows[t]] : 0u;
    int c0 = 0;
#pragma unroll
    for (int t = 0; t < DMAX; ++t) c0 += (t < d) & (f[t] == 0u);
    // quick bound: F <= number of nonzero rows
    const int nz = d - c0;
    if (((mode == CCS_SCORE_COUNT) ? nz : nz - c0) < alpha) return false;
    int F = 0;
#pragma unroll
    for (int a = 0; a < DMAX; ++a) {
        int c = 0;
#pragma unroll
        for (int b = 0; b < DMAX; ++b) c += (b < d) & (f[b] == f[a]);
        F = (a < d && f[a] != 0u && c > F) ? c : F;
    }
    return ((mode == CCS_SCORE_COUNT) ? F : F - c0) >= alpha;
}

// Apply an accepted pair (Alg. 2: x_hat_j <- x_hat_j + omega_j), mark the
// column's rows for the residual phase and, the first time the column turns
// nonzero, enter it in its rows' contributor slots.
__device__ __forceinline__ void apply_pair(const ProblemDev &P, int j, const int32_t *rows, int d,
                                           unsigned long long omega_bits) {
    const double omega = __longlong_as_double((long long)omega_bits);
    P.x_hat[j] = __dadd_rn(__ldcg(P.x_hat + j), omega);
    for (int t = 0; t < d; ++t) P.touched[rows[t]] = 1;
    if (!__ldcg(P.in_slots + j)) {
        P.in_slots[j] = 1;
        for (int t = 0; t < d; ++t) {
            const int pos = atomicAdd(&P.slot_cnt[rows[t]], 1);
            if (pos < kSlots) P.slots[(size_t)rows[t] * kSlots + pos] = j;
        }
    }
}

// r_i = y_i - (sum of the nonzero x_hat_j, j in N(i), in ascending j, from
// +0.0), the residual step of Alg. 2 for one row.
__device__ __forceinline__ double row_residual(const ProblemDev &P, int i) {
    const int cnt = __ldcg(P.slot_cnt + i);
    double s = 0.0;
    if (cnt <= kSlots) {
        // The row's contributors are the columns in its slots (every column
        // with x_hat_j != 0 entered them when it first became nonzero); visit
        // them in ascending j by repeated minimum selection.
        const int32_t *sl = P.slots + (size_t)i * kSlots;
        int js[kSlots];
#pragma unroll
        for (int q = 0; q < kSlots; ++q) js[q] = (q < cnt) ? __ldcg(sl + q) : 0x7fffffff;
        int last = -1;
        for (int step = 0; step < cnt; ++step) {
            int nxt = 0x7fffffff;
#pragma unroll
            for (int q = 0; q < kSlots; ++q) nxt = (js[q] > last && js[q] < nxt) ? js[q] : nxt;
            last = nxt;
            const double v = __ldcg(P.x_hat + nxt);
            if (v != 0.0) s = __dadd_rn(s, v);
        }
    } else {
        // More contributors than slots: walk the whole CSR row.
        const int64_t e = __ldg(P.csr_ptr + i + 1);
        for (int64_t p = __ldg(P.csr_ptr + i); p < e; ++p) {
            const double v = __ldcg(P.x_hat + __ldg(P.csr_cols + p));
            if (v != 0.0) s = __dadd_rn(s, v);
        }
    }
    return __dsub_rn(__ldg(P.y + i), s);
}

}  // namespace ccs
