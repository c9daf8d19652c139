// ccs_device.cuh -- the per-column score and per-row residual, shared by the
// host-driven kernels (ccs_decode.cu) and the persistent engine
// (ccs_engine.cu).
//
// Data read across phases of one persistent launch (r, x_hat, fp, slot
// records, touched, in_slots) is loaded with ld.global.cg (L2, never a
// stale L1 line); the matrix and y are read-only and go through the
// read-only path.
#pragma once

#include "ccs_internal.cuh"

namespace ccs {

// 8-bit fingerprint of a residual entry: 0 exactly when the value is zero
// (+0.0 or -0.0), otherwise a hash of its bits in 1..255.  Equal values have
// equal fingerprints, so a fingerprint count bounds the count of any value.
__device__ __forceinline__ uint8_t fingerprint_of_bits(unsigned long long b) {
    if (b == 0ull) return 0;
    unsigned long long h = (b ^ (b >> 31)) * 0x9e3779b97f4a7c15ull;
    const unsigned f = (unsigned)(h >> 56);
    return (uint8_t)(f == 0u ? 1u : f);
}

__device__ __forceinline__ uint8_t fingerprint(double v) { return fingerprint_of_bits(value_bits(v)); }

// 16-bit fingerprint, same rule: 0 exactly for zero, else a hash in 1..65535.
__device__ __forceinline__ uint16_t fingerprint16_of_bits(unsigned long long b) {
    if (b == 0ull) return 0;
    unsigned long long h = (b ^ (b >> 31)) * 0x9e3779b97f4a7c15ull;
    const unsigned f = (unsigned)(h >> 48);
    return (uint16_t)(f == 0u ? 1u : f);
}

// Store r_i's fingerprint in the problem's width.
__device__ __forceinline__ void store_fp(const ProblemDev &P, int i, double v) {
    if (fp16_for(P.m))
        reinterpret_cast<uint16_t *>(P.fp)[i] = fingerprint16_of_bits(value_bits(v));
    else
        P.fp[i] = fingerprint(v);
}

// Largest multiplicity of a nonzero byte among the first d bytes of the
// packed words w0..w3 (4 bytes each, position t in byte t%4 of word t/4),
// counting each of the d(d-1)/2 pairs once.  Out of line, arguments in
// registers: most columns never need it.
template <int DMAX>
__device__ __noinline__ int fingerprint_max_count(unsigned w0, unsigned w1, unsigned w2,
                                                  unsigned w3, int d) {
    const unsigned w[4] = {w0, w1, w2, w3};
    unsigned f[DMAX];
    int cnt[DMAX];
#pragma unroll
    for (int t = 0; t < DMAX; ++t) {
        f[t] = (w[t >> 2] >> (8 * (t & 3))) & 0xffu;
        cnt[t] = 1;
    }
#pragma unroll
    for (int a = 0; a < DMAX; ++a)
#pragma unroll
        for (int b = a + 1; b < DMAX; ++b) {
            const int e = (b < d) & (f[a] == f[b]);
            cnt[a] += e;
            cnt[b] += e;
        }
    int F = 0;
#pragma unroll
    for (int t = 0; t < DMAX; ++t) F = (t < d && f[t] != 0u && cnt[t] > F) ? cnt[t] : F;
    return F;
}

// Largest multiplicity of a nonzero 16-bit value among the first d halves
// of w0..w7 (position t in half t%2 of word t/2), as above.
template <int DMAX>
__device__ __noinline__ int fingerprint16_max_count(unsigned w0, unsigned w1, unsigned w2,
                                                    unsigned w3, unsigned w4, unsigned w5,
                                                    unsigned w6, unsigned w7, int d) {
    const unsigned w[8] = {w0, w1, w2, w3, w4, w5, w6, w7};
    unsigned f[DMAX];
    int cnt[DMAX];
#pragma unroll
    for (int t = 0; t < DMAX; ++t) {
        f[t] = (w[t >> 1] >> (16 * (t & 1))) & 0xffffu;
        cnt[t] = 1;
    }
#pragma unroll
    for (int a = 0; a < DMAX; ++a)
#pragma unroll
        for (int b = a + 1; b < DMAX; ++b) {
            const int e = (b < d) & (f[a] == f[b]);
            cnt[a] += e;
            cnt[b] += e;
        }
    int F = 0;
#pragma unroll
    for (int t = 0; t < DMAX; ++t) F = (t < d && f[t] != 0u && cnt[t] > F) ? cnt[t] : F;
    return F;
}

// Fingerprints of a column's rows packed for the pair count: kWide selects
// 16-bit values (two a word) over 8-bit ones (four a word).
template <int DMAX, bool kWide>
struct FpWords {
    static constexpr int kWords = kWide ? 8 : 4;
    unsigned w[kWords];
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int q = 0; q < kWords; ++q) w[q] = 0u;
    }
    __device__ __forceinline__ void put(int t, unsigned f) {
        if constexpr (kWide) w[t >> 1] |= f << (16 * (t & 1));
        else w[t >> 2] |= f << (8 * (t & 3));
    }
    __device__ __forceinline__ int max_count(int d) const {
        if constexpr (kWide)
            return fingerprint16_max_count<DMAX>(w[0], w[1], w[2], w[3], w[4], w[5], w[6], w[7], d);
        else
            return fingerprint_max_count<DMAX>(w[0], w[1], w[2], w[3], d);
    }
};

// A row's fingerprint from the shared copy (8- or 16-bit entries).
template <bool kWide>
__device__ __forceinline__ unsigned fp_at(const uint8_t *fp_smem, int row) {
    if constexpr (kWide) return reinterpret_cast<const uint16_t *>(fp_smem)[row];
    else return fp_smem[row];
}

// Exact score from the d gathered values v (value_bits form) -- the
// computation of exact_score without its loads.
template <int DMAX>
__device__ __forceinline__ bool exact_score_values(const unsigned long long (&v)[DMAX], int d,
                                                   int alpha, int mode,
                                                   unsigned long long *omega) {
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

// Shifted variant (Sec. 4.3.1): the only candidate is v[pos], the value at
// the pos-th row of the column (pos = iteration mod d); its count and score
// as in exact_score_values.  A zero candidate is never accepted.
template <int DMAX>
__device__ __forceinline__ bool exact_score_shifted(const unsigned long long (&v)[DMAX], int d,
                                                    int pos, int alpha, int mode,
                                                    unsigned long long *omega) {
    unsigned long long w = 0ull;
#pragma unroll
    for (int t = 0; t < DMAX; ++t) w = (t == pos) ? v[t] : w;
    int c0 = 0, c = 0;
#pragma unroll
    for (int t = 0; t < DMAX; ++t) {
        c0 += (t < d) & (v[t] == 0ull);
        c += (t < d) & (v[t] == w);
    }
    *omega = w;
    if (w == 0ull) return false;
    return ((mode == CCS_SCORE_COUNT) ? c : c - c0) >= alpha;
}

// The fingerprint bound computed from gathered values v (value_bits form):
// false when no value of the column can reach alpha (exact rejection: equal
// values have equal fingerprints).  Cheaper than the O(d^2) compare of
// 64-bit values that it spares most columns.
template <int DMAX>
__device__ __forceinline__ bool values_may_accept(const unsigned long long (&v)[DMAX], int d,
                                                  int alpha, int mode) {
    unsigned w[4] = {0u, 0u, 0u, 0u};
    int c0 = 0;
#pragma unroll
    for (int t = 0; t < DMAX; ++t) {
        const unsigned f = (t < d) ? (unsigned)fingerprint_of_bits(v[t]) : 0u;
        c0 += (t < d) & (v[t] == 0ull);
        w[t >> 2] |= f << (8 * (t & 3));
    }
    const int need = (mode == CCS_SCORE_COUNT) ? alpha : alpha + c0;
    if (d - c0 < need) return false;
    return fingerprint_max_count<DMAX>(w[0], w[1], w[2], w[3], d) >= need;
}

// Exact score of one column from its d row indices `rows` (stride 1).
// Returns true when the pair (j, omega) is accepted; omega's bits in *omega.
// Equality is equality of binary64 values (bit patterns with -0.0 folded);
// the mode is the most frequent nonzero value, ties to the numerically
// smallest (order_key).  Score: Eq. (15) c_omega - c_0, or Alg. 8 c_omega.
// With kPrefilter, before the O(d^2) comparison of 64-bit values the column
// is tested against the fingerprint bound computed from the gathered values
// (equal values have equal fingerprints), which rejects most columns exactly;
// callers whose columns already passed a fingerprint test skip it.
template <int DMAX, bool kPrefilter = true>
__device__ __forceinline__ bool exact_score(const int32_t *rows, int d, const double *r,
                                            int alpha, int mode,
                                            unsigned long long *omega) {
    unsigned long long v[DMAX];
#pragma unroll
    for (int t = 0; t < DMAX; ++t) v[t] = (t < d) ? value_bits(__ldcg(r + rows[t])) : 0ull;
    *omega = 0ull;
    if (kPrefilter && !values_may_accept<DMAX>(v, d, alpha, mode)) return false;
    return exact_score_values<DMAX>(v, d, alpha, mode, omega);
}

// Whether two of a column's nonzero fingerprints f[0..d) are equal.  Zero
// entries and the positions beyond d are replaced by values no fingerprint
// takes (above 16 bits, distinct per position), so one compare per pair
// decides.  Every score needs at least alpha >= 2 equal nonzero values, so a
// column without such a pair is rejected exactly.
template <int DMAX>
__device__ __forceinline__ bool fp_pair_exists(const unsigned (&f)[DMAX], int d) {
    unsigned g[DMAX];
#pragma unroll
    for (int t = 0; t < DMAX; ++t) g[t] = (t < d && f[t] != 0u) ? f[t] : (0x10000u + t);
    bool any = false;
#pragma unroll
    for (int a = 0; a < DMAX; ++a)
#pragma unroll
        for (int b = a + 1; b < DMAX; ++b) any |= (g[a] == g[b]);
    return any;
}

// Largest multiplicity of a nonzero fingerprint among f[0..d).
template <int DMAX, bool kWide>
__device__ __forceinline__ int fp_max_count(const unsigned (&f)[DMAX], int d) {
    FpWords<DMAX, kWide> W;
    W.clear();
#pragma unroll
    for (int t = 0; t < DMAX; ++t) W.put(t, f[t]);
    return W.max_count(d);
}

// Enter column j in the slot records of its d rows: all d slot claims
// (atomicAdd on each record's count) are issued before any column index is
// stored, so the claims travel together instead of one round trip each.
template <int DMAX>
__device__ __forceinline__ void enter_slots(const ProblemDev &P, int j, const int32_t *rows, int d) {
    int pos[DMAX];
#pragma unroll
    for (int t = 0; t < DMAX; ++t)
        pos[t] = (t < d) ? atomicAdd(P.slots + (size_t)rows[t] * kSlotRec, 1) : kSlots;
#pragma unroll
    for (int t = 0; t < DMAX; ++t)
        if (pos[t] < kSlots) P.slots[(size_t)rows[t] * kSlotRec + 1 + pos[t]] = j;
}

// Apply an accepted pair (Alg. 2: x_hat_j <- x_hat_j + omega_j), mark the
// column's rows for the residual phase and, the first time the column turns
// nonzero, enter it in its rows' contributor slots.
template <int DMAX>
__device__ __forceinline__ void apply_pair(const ProblemDev &P, int j, const int32_t *rows, int d,
                                           unsigned long long omega_bits) {
    const double omega = __longlong_as_double((long long)omega_bits);
    P.x_hat[j] = __dadd_rn(__ldcg(P.x_hat + j), omega);
#pragma unroll
    for (int t = 0; t < DMAX; ++t)
        if (t < d) P.touched[rows[t]] = 1;
    if (!__ldcg(P.in_slots + j)) {
        P.in_slots[j] = 1;
        enter_slots<DMAX>(P, j, rows, d);
    }
}

// apply_pair with x_hat_j and the in-slots flag already loaded (issued in the
// same round trip as the column's r gathers).
template <int DMAX>
__device__ __forceinline__ void apply_pair_loaded(const ProblemDev &P, int j, const int32_t *rows,
                                                  int d, unsigned long long omega_bits,
                                                  double xj, uint8_t in_slots) {
    P.x_hat[j] = __dadd_rn(xj, __longlong_as_double((long long)omega_bits));
#pragma unroll
    for (int t = 0; t < DMAX; ++t)
        if (t < d) P.touched[rows[t]] = 1;
    if (!in_slots) {
        P.in_slots[j] = 1;
        enter_slots<DMAX>(P, j, rows, d);
    }
}

// Exponent e of the lowest set bit of a nonzero binary64 value given by its
// bits b (|v| = k 2^e with k odd).
__device__ __forceinline__ int lowbit_exponent(unsigned long long b) {
    const int E = (int)((b >> 52) & 0x7ffull);
    const unsigned long long M = b & 0xfffffffffffffull;
    if (E == 0) return -1074 + __ffsll((long long)M) - 1;
    return E - 1075 + __ffsll((long long)(M | (1ull << 52))) - 1;
}

// Apply an accepted pair while the problem's incremental residual is exact
// (the persistent engine's certificate holds): x_hat_j <- x_hat_j + omega and
// r_i <- r_i - omega on the column's d rows, as binary64 atomic adds into
// r_next.  Every partial result is exact, so the order of the adds does not
// matter and r_next ends equal to y - (ordered sum of the nonzero x_hat).
// The new |x_hat_j| goes into the CTA's running maximum *xmax_s (bits).
template <int DMAX>
__device__ __forceinline__ void apply_exact(const ProblemDev &P, int j, const int32_t *rows, int d,
                                            unsigned long long omega_bits, double xj,
                                            unsigned long long *xmax_s) {
    const double omega = __longlong_as_double((long long)omega_bits);
    const double xn = __dadd_rn(xj, omega);
    P.x_hat[j] = xn;
#pragma unroll
    for (int t = 0; t < DMAX; ++t)
        if (t < d) atomicAdd(P.r_next + rows[t], -omega);
    atomicMax(xmax_s, value_bits(xn) & 0x7fffffffffffffffull);
}

// Ordered row sum from the row's 64-byte slot record js[0..kSlotRec)
// (count, then the columns): the sum of the nonzero x_hat_j, j in N(i), in
// ascending j, from +0.0.
__device__ __forceinline__ double row_sum_from_record(const ProblemDev &P, int i,
                                                      int (&js)[kSlotRec]) {
    const int cnt = js[0];
    double s = 0.0;
    if (cnt <= kSlots) {
        // The row's contributors are the columns in its record (every column
        // with x_hat_j != 0 entered it when it first became nonzero).  Fetch
        // all their x_hat_j at once, then add them in ascending j by repeated
        // minimum selection.
        double v[kSlots];
#pragma unroll
        for (int q = 0; q < kSlots; ++q) {
            js[1 + q] = (q < cnt) ? js[1 + q] : 0x7fffffff;
            v[q] = (q < cnt) ? __ldcg(P.x_hat + js[1 + q]) : 0.0;
        }
        int last = -1;
        for (int step = 0; step < cnt; ++step) {
            int nxt = 0x7fffffff;
            double vn = 0.0;
#pragma unroll
            for (int q = 0; q < kSlots; ++q) {
                const bool take = js[1 + q] > last && js[1 + q] < nxt;
                nxt = take ? js[1 + q] : nxt;
                vn = take ? v[q] : vn;
            }
            last = nxt;
            if (vn != 0.0) s = __dadd_rn(s, vn);
        }
    } else {
        // More contributors than slots: walk the whole CSR row.
        const int64_t e = __ldg(P.csr_ptr + i + 1);
        for (int64_t p = __ldg(P.csr_ptr + i); p < e; ++p) {
            const double xv = __ldcg(P.x_hat + __ldg(P.csr_cols + p));
            if (xv != 0.0) s = __dadd_rn(s, xv);
        }
    }
    return s;
}

__device__ __forceinline__ void load_record(const ProblemDev &P, int i, int (&js)[kSlotRec]) {
    const int4 *rec4 = reinterpret_cast<const int4 *>(P.slots + (size_t)i * kSlotRec);
#pragma unroll
    for (int q = 0; q < kSlotRec / 4; ++q) {
        const int4 v = __ldcg(rec4 + q);
        js[4 * q] = v.x;
        js[4 * q + 1] = v.y;
        js[4 * q + 2] = v.z;
        js[4 * q + 3] = v.w;
    }
}

// Sum of the nonzero x_hat_j over row i's CSR columns in ascending j, from
// +0.0, by the whole warp: the lanes take 32 kU consecutive entries at a
// time and the nonzero values are added chunk by chunk in lane order, so the
// order of the additions is exactly the sequential one.  Only columns whose
// in-slots flag is set are gathered: the flag is a superset of x_hat_j != 0
// (a column sets it the first time it turns nonzero), so a long row with
// few nonzero contributors reads its column indices and flag bytes (which
// stay in L2: the indices stream past with an evict-first load) instead of
// gathering x_hat_j for every entry.  The next 32 kU indices are loaded
// while the current ones are looked up.  Result valid in every lane.
__device__ __forceinline__ double warp_ordered_row_sum_flagged(const ProblemDev &P, int i,
                                                               int lane) {
    constexpr int kU = 16;
    double s = 0.0;
    const int64_t b = __ldg(P.csr_ptr + i), e = __ldg(P.csr_ptr + i + 1);
    int c[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
        const int64_t p = b + 32 * u + lane;
        c[u] = (p < e) ? __ldcs(P.csr_cols + p) : -1;
    }
    for (int64_t p0 = b; p0 < e; p0 += 32 * kU) {
        uint8_t f[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) f[u] = (c[u] >= 0) ? __ldcg(P.in_slots + c[u]) : 0;
        int cn[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int64_t p = p0 + 32 * (kU + u) + lane;
            cn[u] = (p < e) ? __ldcs(P.csr_cols + p) : -1;
        }
        double vj[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) vj[u] = f[u] ? __ldcg(P.x_hat + c[u]) : 0.0;
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            unsigned nz = __ballot_sync(0xffffffffu, value_bits(vj[u]) != 0ull);
            while (nz) {
                const int src = __ffs(nz) - 1;
                nz &= nz - 1;
                s = __dadd_rn(s, __shfl_sync(0xffffffffu, vj[u], src));
            }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) c[u] = cn[u];
    }
    return s;
}

// For the lanes whose row has more contributors than its slot record holds
// (`over`), the row sum by the whole warp, one such row after another; 0.0
// in the other lanes.  Every lane of the warp must call it.  The in-slots
// flags must be current (ordered residual form).
__device__ __forceinline__ double overflow_row_sums(const ProblemDev &P, bool over, int i,
                                                   int lane) {
    double mine = 0.0;
    unsigned ov = __ballot_sync(0xffffffffu, over);
    while (ov) {
        const int src = __ffs(ov) - 1;
        ov &= ov - 1;
        const int row = __shfl_sync(0xffffffffu, i, src);
        const double s = warp_ordered_row_sum_flagged(P, row, lane);
        if (lane == src) mine = s;
    }
    return mine;
}

// r_i = y_i - (sum of the nonzero x_hat_j, j in N(i), in ascending j, from
// +0.0), the residual step of Alg. 2 for one row.
__device__ __forceinline__ double row_residual(const ProblemDev &P, int i) {
    int js[kSlotRec];
    load_record(P, i, js);
    return __dsub_rn(__ldg(P.y + i), row_sum_from_record(P, i, js));
}

}  // namespace ccs
