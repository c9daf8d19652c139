// ccs_setup.cu -- expander generation, CSR transpose and y = A x.
//
// Generation follows the Sec. 1.1 footnote of the paper: columns are drawn
// independently, each column's support uniform over the C(m, d) subsets of
// size d.  Every column owns a counter-based SplitMix64 stream, so a column
// is one thread's work and the matrix depends only on (n, m, d, seed).
#include <cstdarg>
#include <cstdio>

#include "ccs_checks.cuh"
#include "ccs_internal.cuh"

namespace ccs {

// ---------------------------------------------------------------------------
// Random numbers
// ---------------------------------------------------------------------------

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): Weyl increment
// 0x9e3779b97f4a7c15, then the variant-13 mixing function.
__device__ __forceinline__ uint64_t splitmix64(uint64_t &state) {
    state += 0x9e3779b97f4a7c15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Lemire's bounded draw (ACM TOMACS 2019): high word of x * range, redrawing
// while the low word is below 2^64 mod range.
__device__ __forceinline__ uint32_t draw_below(uint64_t &state, uint32_t range) {
    uint64_t x = splitmix64(state);
    uint64_t lo = x * (uint64_t)range;
    uint64_t hi = __umul64hi(x, (uint64_t)range);
    if (lo < range) {
        const uint64_t floor_mod = (0ull - (uint64_t)range) % (uint64_t)range;
        while (lo < floor_mod) {
            x = splitmix64(state);
            lo = x * (uint64_t)range;
            hi = __umul64hi(x, (uint64_t)range);
        }
    }
    return (uint32_t)hi;
}

// One thread per column: d distinct rows, sorted ascending.
__global__ void k_generate_columns(int n, int m, int d, uint64_t seed, int32_t *csc_rows) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    uint64_t state = seed + (uint64_t)(j + 1) * 0xd1b54a32d192ed03ull;
    int32_t rows[kMaxD];
    int got = 0;
    while (got < d) {
        const int32_t row = (int32_t)draw_below(state, (uint32_t)m);
        bool seen = false;
        for (int t = 0; t < got; ++t) seen |= (rows[t] == row);
        if (!seen) rows[got++] = row;
    }
    for (int a = 1; a < d; ++a) {
        const int32_t v = rows[a];
        int b = a - 1;
        while (b >= 0 && rows[b] > v) {
            rows[b + 1] = rows[b];
            --b;
        }
        rows[b + 1] = v;
    }
    int32_t *out = csc_rows + (size_t)j * d;
    for (int t = 0; t < d; ++t) out[t] = rows[t];
}

// ---------------------------------------------------------------------------
// CSR transpose: count -> scan -> scatter -> sort each row
// ---------------------------------------------------------------------------

__global__ void k_count_rows(long long edges, const int32_t *csc_rows, int32_t *deg) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < edges;
         e += (long long)gridDim.x * blockDim.x)
        atomicAdd(&deg[csc_rows[e]], 1);
}

constexpr int kScanBlock = 1024;

// Per block of kScanBlock rows: inclusive prefix of deg into ptr[1 + i],
// block total into sums[block], largest degree into *max_deg.
__global__ void __launch_bounds__(kScanBlock)
k_scan_local(int m, const int32_t *deg, int64_t *ptr, int64_t *sums, int *max_deg) {
    __shared__ long long warp_tot[kScanBlock / 32];
    const int i = blockIdx.x * kScanBlock + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long v = (i < m) ? deg[i] : 0;
    int mx = (int)v;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0 && mx > 0) atomicMax(max_deg, mx);
    long long inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        long long w = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        warp_tot[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    if (warp > 0) inc += warp_tot[warp - 1];
    if (i < m) ptr[i + 1] = inc;
    if (threadIdx.x == kScanBlock - 1) sums[blockIdx.x] = inc;
}

// Exclusive scan of the block totals, one block, sequential over chunks.
__global__ void __launch_bounds__(1024) k_scan_sums(int nblocks, int64_t *sums) {
    __shared__ long long warp_tot[32];
    __shared__ long long carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nblocks; base += 1024) {
        const int i = base + threadIdx.x;
        long long v = (i < nblocks) ? sums[i] : 0;
        long long inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) warp_tot[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            long long w = warp_tot[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                long long t = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += t;
            }
            warp_tot[lane] = w;
        }
        __syncthreads();
        if (warp > 0) inc += warp_tot[warp - 1];
        const long long c = carry;
        if (i < nblocks) sums[i] = c + inc - v;  // exclusive
        __syncthreads();
        if (threadIdx.x == 1023) carry = c + inc;
        __syncthreads();
    }
}

__global__ void k_scan_add(int m, int64_t *ptr, const int64_t *sums) {
    const int i = blockIdx.x * kScanBlock + threadIdx.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) ptr[0] = 0;
    if (i < m) ptr[i + 1] += sums[blockIdx.x];
}

__global__ void k_scatter_cols(int n, int d, const int32_t *csc_rows, const int64_t *ptr,
                               int32_t *fill, int32_t *csr_cols) {
    const long long edges = (long long)n * d;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < edges;
         e += (long long)gridDim.x * blockDim.x) {
        const int32_t i = csc_rows[e];
        const int32_t pos = atomicAdd(&fill[i], 1);
        csr_cols[ptr[i] + pos] = (int32_t)(e / d);
    }
}

// One block per row: bitonic sort of the row's columns in shared memory
// (padded with INT_MAX to `cap`, a power of two).
__global__ void k_sort_rows(int m, int cap, const int64_t *ptr, int32_t *csr_cols) {
    extern __shared__ int32_t buf[];
    for (int i = blockIdx.x; i < m; i += gridDim.x) {
        const int64_t b = ptr[i];
        const int len = (int)(ptr[i + 1] - b);
        if (len > 1) {
            int size = 2;
            while (size < len) size <<= 1;
            for (int t = threadIdx.x; t < size; t += blockDim.x)
                buf[t] = t < len ? csr_cols[b + t] : 0x7fffffff;
            __syncthreads();
            for (int k = 2; k <= size; k <<= 1) {
                for (int jj = k >> 1; jj > 0; jj >>= 1) {
                    for (int t = threadIdx.x; t < size; t += blockDim.x) {
                        const int p = t ^ jj;
                        if (p > t) {
                            const bool up = (t & k) == 0;
                            const int32_t a = buf[t], c = buf[p];
                            if ((a > c) == up) {
                                buf[t] = c;
                                buf[p] = a;
                            }
                        }
                    }
                    __syncthreads();
                }
            }
            for (int t = threadIdx.x; t < len; t += blockDim.x) csr_cols[b + t] = buf[t];
            __syncthreads();
        }
    }
    (void)cap;
}

// Rows of at most 32 E columns: one warp a row, the row in registers (E per
// lane, element lane * E + e), bitonic sort by register exchanges and warp
// shuffles: no shared memory and no block barriers.
template <int E>
__global__ void k_sort_rows_warp(int m, const int64_t *ptr, int32_t *csr_cols) {
    constexpr int kCap = 32 * E;
    const int lane = threadIdx.x & 31;
    const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = w0; i < m; i += nw) {
        const int64_t b = ptr[i];
        const int len = (int)(ptr[i + 1] - b);
        if (len <= 1) continue;
        int32_t v[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int idx = lane * E + e;
            v[e] = idx < len ? csr_cols[b + idx] : 0x7fffffff;
        }
#pragma unroll
        for (int k = 2; k <= kCap; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                if (j < E) {
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const int p = e ^ j;
                        if (p > e) {
                            const bool up = ((lane * E + e) & k) == 0;
                            const int32_t a = v[e], c = v[p];
                            if ((a > c) == up) {
                                v[e] = c;
                                v[p] = a;
                            }
                        }
                    }
                } else {
                    const int lj = j / E;
                    const bool lower = (lane & lj) == 0;
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const int32_t o = __shfl_xor_sync(0xffffffffu, v[e], lj);
                        const bool up = ((lane * E + e) & k) == 0;
                        v[e] = (lower == up) ? min(v[e], o) : max(v[e], o);
                    }
                }
            }
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int idx = lane * E + e;
            if (idx < len) csr_cols[b + idx] = v[e];
        }
    }
}

// ---------------------------------------------------------------------------
// y = A x: one warp per row, ascending column order
// ---------------------------------------------------------------------------

// Sum of v[j] over the row's columns in ascending j, from +0.0, skipping zero
// entries.  The 32 lanes fetch 32 consecutive entries at a time; the nonzero
// ones are then added in lane order, so the addition order is exactly the
// sequential one.  Result valid in every lane.
__device__ __forceinline__ double warp_ordered_row_sum(const int64_t *ptr, const int32_t *cols,
                                                       const double *v, int i, int lane) {
    double s = 0.0;
    const int64_t b = ptr[i], e = ptr[i + 1];
    for (int64_t p0 = b; p0 < e; p0 += 32) {
        const int64_t p = p0 + lane;
        const double vj = (p < e) ? v[cols[p]] : 0.0;
        unsigned nz = __ballot_sync(0xffffffffu, vj != 0.0);
        while (nz) {
            const int src = __ffs(nz) - 1;
            nz &= nz - 1;
            s = __dadd_rn(s, __shfl_sync(0xffffffffu, vj, src));
        }
    }
    return s;
}

// Column scales for signals that are not dissociated (Sec. 4.3.3): one
// i.i.d. scale per column, uniform on [1, 2) to a grid of 2^-20 -- 1 plus the
// top 20 bits of the first draw of the column's SplitMix64 stream, times
// 2^-20 (exact in binary64).
__global__ void k_column_scales(int n, uint64_t seed, double *s) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x) {
        uint64_t state = seed + (uint64_t)(j + 1) * 0xd1b54a32d192ed03ull;
        const uint64_t k = splitmix64(state) >> 44;
        s[j] = __dadd_rn(1.0, (double)k * 0x1p-20);
    }
}

// y = A diag(s) x: the row's nonzero products s_j x_j (each rounded once),
// added in ascending j from +0.0 by the whole warp.
__global__ void k_measure_scaled(int m, const int64_t *ptr, const int32_t *cols,
                                 const double *sc, const double *x, double *y) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < m; i += warps) {
        double s = 0.0;
        const int64_t b = ptr[i], e = ptr[i + 1];
        for (int64_t p0 = b; p0 < e; p0 += 32) {
            const int64_t p = p0 + lane;
            const int c = (p < e) ? cols[p] : 0;
            const double vj = (p < e) ? __dmul_rn(sc[c], x[c]) : 0.0;
            unsigned nz = __ballot_sync(0xffffffffu, vj != 0.0);
            while (nz) {
                const int src = __ffs(nz) - 1;
                nz &= nz - 1;
                s = __dadd_rn(s, __shfl_sync(0xffffffffu, vj, src));
            }
        }
        if (lane == 0) y[i] = s;
    }
}

// x_j = z_j / s_j (the decode of a column-scaled measurement is z = s . x).
__global__ void k_unscale(int n, const double *sc, const double *z, double *x) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x)
        x[j] = __ddiv_rn(z[j], sc[j]);
}

__global__ void k_measure(int m, const int64_t *ptr, const int32_t *cols, const double *x,
                          double *y) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < m; i += warps) {
        const double s = warp_ordered_row_sum(ptr, cols, x, i, lane);
        if (lane == 0) y[i] = s;
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

static thread_local char g_last_error[512] = "";

void set_last_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
}

int cuda_fail(cudaError_t e, const char *what) {
    set_last_error("%s: %s", what, cudaGetErrorString(e));
    return CCS_ECUDA;
}

int check_sizes(int32_t n, int32_t m, int32_t d) {
    if (n < 1 || m < 1 || d < 1 || d > kMaxD || d > m) {
        set_last_error("invalid sizes n=%d m=%d d=%d (need n,m >= 1, 1 <= d <= min(m, %d))",
                       n, m, d, kMaxD);
        return CCS_EINVAL;
    }
    if ((long long)n * d >= (1ll << 31)) {
        set_last_error("n*d = %lld exceeds the int32 edge index range", (long long)n * d);
        return CCS_EINVAL;
    }
    return CCS_OK;
}

int check_aligned(const char *who, const char *what, const void *p, unsigned align) {
    if (reinterpret_cast<uintptr_t>(p) % align) {
        set_last_error("%s: %s is not on a %u-byte boundary", who, what, align);
        return CCS_EINVAL;
    }
    return CCS_OK;
}

int check_problem_arrays(const char *who, const int32_t *csc_rows, const int64_t *csr_ptr,
                         const int32_t *csr_cols, const double *y, const double *x_hat,
                         const double *r, const int64_t *r0_hist) {
    int rc;
    if ((rc = check_aligned(who, "csc_rows", csc_rows, 16))) return rc;
    if ((rc = check_aligned(who, "csr_ptr", csr_ptr, 8))) return rc;
    if ((rc = check_aligned(who, "csr_cols", csr_cols, 4))) return rc;
    if ((rc = check_aligned(who, "y", y, 8))) return rc;
    if ((rc = check_aligned(who, "x_hat", x_hat, 8))) return rc;
    if ((rc = check_aligned(who, "r", r, 8))) return rc;
    return check_aligned(who, "r0_hist", r0_hist, 8);
}

static size_t make_expander_ws(int32_t n, int32_t m) {
    (void)n;
    const size_t nblocks = ((size_t)m + kScanBlock - 1) / kScanBlock;
    return align_up((size_t)m * 4, 256) + align_up(nblocks * 8, 256) + 256;
}

static int grid_for(long long work, int block) {
    long long g = (work + block - 1) / block;
    if (g > 152ll * 32) g = 152ll * 32;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace ccs

using namespace ccs;

extern "C" {

const char *ccs_last_error(void) { return g_last_error; }

int ccs_version(void) { return 10000; }

const char *ccs_status_string(int status) {
    switch (status) {
        case CCS_OK: return "CCS_OK";
        case CCS_EINVAL: return "CCS_EINVAL";
        case CCS_ENOMEM: return "CCS_ENOMEM";
        case CCS_ECUDA: return "CCS_ECUDA";
        case CCS_ETIMEOUT: return "CCS_ETIMEOUT";
        case CCS_EBUDGET: return "CCS_EBUDGET";
        case CCS_EBUSY: return "CCS_EBUSY";
        default: return "CCS_E?";
    }
}

void ccs_params_init(ccs_params *p) {
    if (!p) return;
    p->alpha = 2;
    p->max_iter = 100;
    p->score_mode = CCS_SCORE_L0_DECREASE;
    p->engine = CCS_ENGINE_AUTO;
    p->watchdog_ms = 0;
    p->debug_flags = 0;
    p->schedule = 0;
    p->shifted = 0;
}

size_t ccs_workspace_size(int32_t op, int32_t n, int32_t m, int32_t d) {
    if (check_sizes(n, m, d) != CCS_OK) return 0;
    if (op == CCS_OP_MAKE_EXPANDER) return make_expander_ws(n, m);
    if (op == CCS_OP_DECODE) return engine_header_bytes(1) + decode_ws_layout(n, m, nullptr, nullptr);
    return 0;
}

}  // extern "C"

namespace ccs {

// First part of the expander's construction, all enqueued on `s`: the
// columns, the row degrees and their prefix (csr_ptr), the CSR scatter.
// *max_deg_dev receives the device address of the largest row degree, which
// sizes the row sort (expander_sort_rows).  Arguments already checked.
int expander_build_async(int32_t n, int32_t m, int32_t d, uint64_t seed, int32_t *csc_rows,
                         int64_t *csr_ptr, int32_t *csr_cols, void *ws, cudaStream_t s,
                         int **max_deg_dev) {
    char *base = static_cast<char *>(ws);
    int32_t *deg = reinterpret_cast<int32_t *>(base);
    const int nblocks = (m + kScanBlock - 1) / kScanBlock;
    int64_t *sums = reinterpret_cast<int64_t *>(base + align_up((size_t)m * 4, 256));
    int *max_deg = reinterpret_cast<int *>(base + align_up((size_t)m * 4, 256) +
                                           align_up((size_t)nblocks * 8, 256));
    const long long edges = (long long)n * d;

    k_generate_columns<<<(n + 255) / 256, 256, 0, s>>>(n, m, d, seed, csc_rows);
    CCS_CUDA_TRY(cudaGetLastError());
    CCS_CUDA_TRY(cudaMemsetAsync(deg, 0, (size_t)m * 4, s));
    CCS_CUDA_TRY(cudaMemsetAsync(max_deg, 0, sizeof(int), s));
    k_count_rows<<<grid_for(edges, 256), 256, 0, s>>>(edges, csc_rows, deg);
    k_scan_local<<<nblocks, kScanBlock, 0, s>>>(m, deg, csr_ptr, sums, max_deg);
    k_scan_sums<<<1, 1024, 0, s>>>(nblocks, sums);
    k_scan_add<<<nblocks, kScanBlock, 0, s>>>(m, csr_ptr, sums);
    CCS_CUDA_TRY(cudaGetLastError());
    CCS_CUDA_TRY(cudaMemsetAsync(deg, 0, (size_t)m * 4, s));
    k_scatter_cols<<<grid_for(edges, 256), 256, 0, s>>>(n, d, csc_rows, csr_ptr, deg, csr_cols);
    CCS_CUDA_TRY(cudaGetLastError());
    *max_deg_dev = max_deg;
    return CCS_OK;
}

// Second part: sort every CSR row ascending, given the largest row degree
// (read back from expander_build_async).  CCS_EINVAL when a row is longer
// than the on-chip sort takes.  Enqueued on `s`.
int expander_sort_rows(int32_t m, int64_t *csr_ptr, int32_t *csr_cols, int host_max,
                       cudaStream_t s) {
    if (host_max > kMaxSortRow) {
        set_last_error("ccs_make_expander: a row has %d columns (limit %d)", host_max,
                       kMaxSortRow);
        return CCS_EINVAL;
    }
    if (host_max > 1 && host_max <= 1024) {
        // rows of at most 1024 columns: a warp a row, in registers
        int cap = 32;
        while (cap < host_max) cap <<= 1;
        const int grid = 152 * 16, threads = 256;
        switch (cap) {
            case 32: k_sort_rows_warp<1><<<grid, threads, 0, s>>>(m, csr_ptr, csr_cols); break;
            case 64: k_sort_rows_warp<2><<<grid, threads, 0, s>>>(m, csr_ptr, csr_cols); break;
            case 128: k_sort_rows_warp<4><<<grid, threads, 0, s>>>(m, csr_ptr, csr_cols); break;
            case 256: k_sort_rows_warp<8><<<grid, threads, 0, s>>>(m, csr_ptr, csr_cols); break;
            case 512: k_sort_rows_warp<16><<<grid, threads, 0, s>>>(m, csr_ptr, csr_cols); break;
            default: k_sort_rows_warp<32><<<grid, threads, 0, s>>>(m, csr_ptr, csr_cols); break;
        }
        CCS_CUDA_TRY(cudaGetLastError());
    } else if (host_max > 1) {
        int cap = 2;
        while (cap < host_max) cap <<= 1;
        const size_t smem = (size_t)cap * 4;
        if (smem > 48 * 1024)
            CCS_CUDA_TRY(cudaFuncSetAttribute(k_sort_rows,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem));
        const int threads = cap >= 1024 ? 1024 : (cap < 32 ? 32 : cap);
        const int grid = m < 152 * 16 ? m : 152 * 16;
        k_sort_rows<<<grid, threads, smem, s>>>(m, cap, csr_ptr, csr_cols);
        CCS_CUDA_TRY(cudaGetLastError());
    }
    return CCS_OK;
}

}  // namespace ccs

extern "C" {

int ccs_make_expander(int32_t n, int32_t m, int32_t d, uint64_t seed, int32_t *csc_rows,
                      int64_t *csr_ptr, int32_t *csr_cols, void *ws, size_t ws_bytes,
                      ccs_stream_t stream) {
    int rc = check_sizes(n, m, d);
    if (rc) return rc;
    if (!csc_rows || !csr_ptr || !csr_cols || !ws) {
        set_last_error("ccs_make_expander: null pointer argument");
        return CCS_EINVAL;
    }
    if (ws_bytes < make_expander_ws(n, m)) {
        set_last_error("ccs_make_expander: workspace %zu < %zu bytes", ws_bytes,
                       make_expander_ws(n, m));
        return CCS_ENOMEM;
    }
    if ((rc = check_problem_arrays("ccs_make_expander", csc_rows, csr_ptr, csr_cols, nullptr,
                                   nullptr, nullptr, nullptr)) ||
        (rc = check_aligned("ccs_make_expander", "ws", ws, kWorkspaceAlign)))
        return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int *max_deg = nullptr;
    if ((rc = expander_build_async(n, m, d, seed, csc_rows, csr_ptr, csr_cols, ws, s, &max_deg)))
        return rc;
    int host_max = 0;
    CCS_CUDA_TRY(cudaMemcpyAsync(&host_max, max_deg, sizeof(int), cudaMemcpyDeviceToHost, s));
    CCS_CUDA_TRY(cudaStreamSynchronize(s));
    if ((rc = expander_sort_rows(m, csr_ptr, csr_cols, host_max, s))) return rc;
    CCS_CUDA_TRY(cudaStreamSynchronize(s));
    return CCS_OK;
}

int ccs_measure(int32_t n, int32_t m, int32_t d, const int64_t *csr_ptr,
                const int32_t *csr_cols, const double *x, double *y, ccs_stream_t stream) {
    int rc = check_sizes(n, m, d);
    if (rc) return rc;
    if (!csr_ptr || !csr_cols || !x || !y) {
        set_last_error("ccs_measure: null pointer argument");
        return CCS_EINVAL;
    }
    if ((rc = check_problem_arrays("ccs_measure", nullptr, csr_ptr, csr_cols, y, nullptr,
                                   nullptr, nullptr)) ||
        (rc = check_aligned("ccs_measure", "x", x, 8)))
        return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const long long threads = (long long)m * 32;
    k_measure<<<grid_for(threads, 256), 256, 0, s>>>(m, csr_ptr, csr_cols, x, y);
    CCS_CUDA_TRY(cudaGetLastError());
    return CCS_OK;
}

int ccs_column_scales(int32_t n, uint64_t seed, double *scales, ccs_stream_t stream) {
    if (n < 1 || !scales) {
        set_last_error("ccs_column_scales: n < 1 or null output");
        return CCS_EINVAL;
    }
    if (int rc = check_aligned("ccs_column_scales", "s", scales, 8)) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    k_column_scales<<<grid_for(n, 256), 256, 0, s>>>(n, seed, scales);
    CCS_CUDA_TRY(cudaGetLastError());
    return CCS_OK;
}

int ccs_measure_scaled(int32_t n, int32_t m, int32_t d, const int64_t *csr_ptr,
                       const int32_t *csr_cols, const double *scales, const double *x,
                       double *y, ccs_stream_t stream) {
    int rc = check_sizes(n, m, d);
    if (rc) return rc;
    if (!csr_ptr || !csr_cols || !scales || !x || !y) {
        set_last_error("ccs_measure_scaled: null pointer argument");
        return CCS_EINVAL;
    }
    if ((rc = check_problem_arrays("ccs_measure_scaled", nullptr, csr_ptr, csr_cols, y, nullptr,
                                   nullptr, nullptr)) ||
        (rc = check_aligned("ccs_measure_scaled", "x", x, 8)) ||
        (rc = check_aligned("ccs_measure_scaled", "s", scales, 8)))
        return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const long long threads = (long long)m * 32;
    k_measure_scaled<<<grid_for(threads, 256), 256, 0, s>>>(m, csr_ptr, csr_cols, scales, x, y);
    CCS_CUDA_TRY(cudaGetLastError());
    return CCS_OK;
}

int ccs_unscale(int32_t n, const double *scales, const double *z, double *x,
                ccs_stream_t stream) {
    if (n < 1 || !scales || !z || !x) {
        set_last_error("ccs_unscale: n < 1 or null pointer argument");
        return CCS_EINVAL;
    }
    int rc;
    if ((rc = check_aligned("ccs_unscale", "s", scales, 8)) ||
        (rc = check_aligned("ccs_unscale", "z", z, 8)) ||
        (rc = check_aligned("ccs_unscale", "x", x, 8)))
        return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    k_unscale<<<grid_for(n, 256), 256, 0, s>>>(n, scales, z, x);
    CCS_CUDA_TRY(cudaGetLastError());
    return CCS_OK;
}

}  // extern "C"
