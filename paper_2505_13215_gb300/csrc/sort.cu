// sort.cu -- Alg. 1 CreateTiles, DuplicateWithKeys, SortByKeys and
// IdentifyTileRanges.
//
// The instance key is (global tile index, camera depth) and the sort is a
// stable LSD radix sort of it.  Every instance of one projected row carries
// the same depth, so the depth digits (the least significant ones) are sorted
// once per row, before duplication: rows are radix-sorted by the IEEE bits
// of their depth (positive floats order like their bit patterns), the
// instances are emitted in that row order, and the tile digits are then
// radix-sorted stably.  The result is the order of a stable sort of the full
// key in emission order.
//
// Radix passes are single-pass "onesweep"-style: one 8-bit digit per pass,
// partitions of 3840 keys taken in ticket order by persistent CTAs, local
// ranking with warp match + shared-memory counters, and a decoupled look-back
// across partitions whose waits are bounded (SPLAT_ERR_TIMEOUT on expiry).
#include <algorithm>

#include "splat_internal.cuh"

namespace splat {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 15;
constexpr int kSortPart = kSortThreads * kSortItems;  // keys per partition
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanPart = kScanThreads * kScanItems;
constexpr int kDupChunk = 2048;  // instance slots per duplicate work item
constexpr int kDupThreads = 256;

constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagPrefix = 2u << 30;
constexpr uint32_t kValMask = (1u << 30) - 1;

// Exclusive scan of one value per thread across a 256-thread block.
__device__ __forceinline__ uint32_t block_excl_scan256(uint32_t v, uint32_t* s_tmp, uint32_t* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_tmp[warp] = x;
    __syncthreads();
    uint32_t wsum = 0, all = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const uint32_t t = s_tmp[w];
        if (w < warp) wsum += t;
        all += t;
    }
    __syncthreads();
    if (total) *total = all;
    return wsum + x - v;
}

// ---------------------------------------------------------------------------
// Depth keys of the projected rows + histograms of their 4 digits
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_depth_keys(splat_proj proj, int64_t n_rows, uint32_t* keys, uint32_t* vals,
                                                    uint32_t* hist /*[4][256]*/, uint32_t* zero_a, int64_t n_zero_a,
                                                    unsigned long long* zero_b, int64_t n_zero_b)
{
    __shared__ uint32_t s_hist[4][kRadix];
    for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) (&s_hist[0][0])[i] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_rows; r += stride) {
        const uint32_t nt = proj.n_tiles[r];
        const float depth = ((const float4*)proj.rgb_depth)[r].w;
        const uint32_t k = nt > 0 ? __float_as_uint(depth) : 0xffffffffu;
        keys[r] = k;
        vals[r] = (uint32_t)r;
#pragma unroll
        for (int p = 0; p < 4; ++p) atomicAdd(&s_hist[p][(k >> (8 * p)) & 0xff], 1u);
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_zero_a; i += stride) zero_a[i] = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_zero_b; i += stride) zero_b[i] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) {
        const uint32_t c = (&s_hist[0][0])[i];
        if (c) atomicAdd(&hist[i], c);
    }
}

// ---------------------------------------------------------------------------
// One onesweep radix pass (8-bit digit at `shift`)
// ---------------------------------------------------------------------------

struct PassArgs {
    const uint32_t* keys_in;
    const uint32_t* vals_in;
    uint32_t* keys_out;  // may be null (keys not needed after this pass)
    uint32_t* vals_out;
    const int64_t* n_dev;  // element count on the device (null: n_host)
    int64_t n_host;
    int64_t cap;
    const uint32_t* hist;  // [256] digit counts of this pass
    uint32_t* lb;          // [parts][256] look-back words of this pass (zeroed)
    uint32_t* lb_next;     // [parts][256] zeroed here for the next pass (may be null)
    uint32_t* ticket;
    int32_t* status;
    int stage;
    int shift;
    int64_t spin_limit;
};

__global__ void __launch_bounds__(kSortThreads) k_onesweep(PassArgs a)
{
    __shared__ uint32_t s_keys[kSortPart];
    __shared__ uint32_t s_vals[kSortPart];
    __shared__ uint32_t s_whist[kSortWarps][kRadix];
    __shared__ uint32_t s_gofs[kRadix];
    __shared__ uint32_t s_dstart[kRadix];
    __shared__ uint32_t s_base[kRadix];
    __shared__ uint32_t s_tmp[8];
    __shared__ int64_t s_ticket;

    if (status_failed(a.status)) return;
    const int64_t n = a.n_dev ? min(*a.n_dev, a.cap) : a.n_host;
    if (n <= 0) return;
    const int64_t parts = (n + kSortPart - 1) / kSortPart;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = lanemask_lt();
    s_gofs[tid] = block_excl_scan256(a.hist[tid], s_tmp, nullptr);

    for (;;) {
        if (tid == 0) s_ticket = atomicAdd(a.ticket, 1u);
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) s_whist[w][tid] = 0;
        __syncthreads();
        const int64_t ticket = s_ticket;
        if (ticket >= parts) break;
        const int64_t base = ticket * kSortPart;
        const int64_t wbase = base + (int64_t)warp * 32 * kSortItems;

        uint32_t k[kSortItems], v[kSortItems], r[kSortItems];
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const int64_t idx = wbase + j * 32 + lane;
            const bool ok = idx < n;
            k[j] = ok ? a.keys_in[idx] : 0u;
            v[j] = ok ? a.vals_in[idx] : 0u;
        }
        // warp-level stable ranking, items in (j, lane) order
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const int64_t idx = wbase + j * 32 + lane;
            const bool ok = idx < n;
            const unsigned valid = __ballot_sync(0xffffffffu, ok);
            r[j] = 0;
            if (ok) {
                const uint32_t d = (k[j] >> a.shift) & 0xff;
                const unsigned peers = __match_any_sync(valid, d);
                const int leader = __ffs(peers) - 1;
                uint32_t prev = 0;
                if (lane == leader) {
                    prev = s_whist[warp][d];
                    s_whist[warp][d] = prev + __popc(peers);
                }
                prev = __shfl_sync(peers, prev, leader);
                r[j] = prev + __popc(peers & lt);
            }
            __syncwarp();
        }
        __syncthreads();
        // per digit: exclusive prefix over warps, partition count
        const int d = tid;
        uint32_t cnt = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t c = s_whist[w][d];
            s_whist[w][d] = cnt;
            cnt += c;
        }
        uint32_t* my = a.lb + ticket * kRadix + d;
        st_relaxed(my, (ticket == 0 ? kFlagPrefix : kFlagAgg) | cnt);
        if (a.lb_next) a.lb_next[ticket * kRadix + d] = 0;
        s_dstart[d] = block_excl_scan256(cnt, s_tmp, nullptr);
        // decoupled look-back for digit d
        uint32_t excl = 0;
        if (ticket > 0) {
            int64_t j = ticket - 1;
            int64_t spins = 0;
            for (;;) {
                const uint32_t s = ld_relaxed(a.lb + j * kRadix + d);
                const uint32_t flag = s & ~kValMask;
                if (flag == 0) {
                    if (++spins > a.spin_limit) {
                        set_status(a.status, SPLAT_ERR_TIMEOUT, a.stage, ticket);
                        break;
                    }
                    if (spins > 64) __nanosleep(64);
                    continue;
                }
                excl += s & kValMask;
                if (flag == kFlagPrefix || j == 0) break;
                --j;
            }
            st_relaxed(my, kFlagPrefix | ((excl + cnt) & kValMask));
        }
        s_base[d] = s_gofs[d] + excl - s_dstart[d];
        __syncthreads();
        // local scatter into digit order
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const int64_t idx = wbase + j * 32 + lane;
            if (idx < n) {
                const uint32_t dd = (k[j] >> a.shift) & 0xff;
                const uint32_t pos = s_dstart[dd] + s_whist[warp][dd] + r[j];
                s_keys[pos] = k[j];
                s_vals[pos] = v[j];
            }
        }
        __syncthreads();
        const int nvalid = (int)min((int64_t)kSortPart, n - base);
        for (int i = tid; i < nvalid; i += kSortThreads) {
            const uint32_t key = s_keys[i];
            const uint32_t out = s_base[(key >> a.shift) & 0xff] + i;
            if (out >= (uint64_t)n) continue;  // only after a timed-out look-back
            if (a.keys_out) a.keys_out[out] = key;
            a.vals_out[out] = s_vals[i];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Exclusive scan of the tile counts in depth order (A5) + chunk starts for
// the load-balanced duplication + capacity check.
// ---------------------------------------------------------------------------

struct ScanArgs {
    const uint32_t* rows;      // [n_rows] depth-sorted rows
    const uint32_t* n_tiles;   // [n_rows] per row
    int64_t n_rows;
    uint32_t* offsets;         // [n_rows] exclusive prefix (saturated at 2^32-1)
    uint32_t* chunk_row;       // [n_chunks_max] first sorted position of each duplicate chunk
    int64_t n_chunks_max;
    unsigned long long* lb;    // [parts] look-back words (zeroed)
    uint32_t* ticket;
    int64_t* n_instances;      // out: K
    int64_t capacity;
    int32_t* status;
    int64_t spin_limit;
};

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(ScanArgs a)
{
    __shared__ uint32_t s_tmp[8];
    __shared__ int64_t s_ticket;
    __shared__ unsigned long long s_excl;
    constexpr unsigned long long kA = 1ull << 62, kP = 2ull << 62, kM = (1ull << 62) - 1;
    if (status_failed(a.status)) return;  // the row order is not valid after a failed sort
    const int64_t parts = (a.n_rows + kScanPart - 1) / kScanPart;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_ticket = atomicAdd(a.ticket, 1u);
        __syncthreads();
        const int64_t ticket = s_ticket;
        if (ticket >= parts) break;
        const int64_t base = ticket * kScanPart;
        unsigned long long local[kScanItems];
        unsigned long long running = 0;  // total of the earlier rounds of this partition
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            const int64_t idx = base + (int64_t)j * kScanThreads + tid;
            const uint32_t c = idx < a.n_rows ? a.n_tiles[a.rows[idx]] : 0u;
            uint32_t tot;
            const uint32_t ex = block_excl_scan256(c, s_tmp, &tot);
            local[j] = running + ex;
            running += tot;
        }
        const unsigned long long agg = running;
        if (tid == 0) {
            unsigned long long excl = 0;
            st_relaxed64(a.lb + ticket, (ticket == 0 ? kP : kA) | agg);
            if (ticket > 0) {
                int64_t j = ticket - 1, spins = 0;
                for (;;) {
                    const unsigned long long s = ld_relaxed64(a.lb + j);
                    const unsigned long long flag = s & ~kM;
                    if (flag == 0) {
                        if (++spins > a.spin_limit) {
                            set_status(a.status, SPLAT_ERR_TIMEOUT, SPLAT_STAGE_SCAN, ticket);
                            break;
                        }
                        if (spins > 64) __nanosleep(64);
                        continue;
                    }
                    excl += s & kM;
                    if (flag == kP || j == 0) break;
                    --j;
                }
                st_relaxed64(a.lb + ticket, kP | ((excl + agg) & kM));
            }
            s_excl = excl;
            if (ticket == parts - 1) {
                const int64_t K = (int64_t)(excl + agg);
                *a.n_instances = K;
                if (K > a.capacity) set_status(a.status, SPLAT_ERR_CAPACITY, SPLAT_STAGE_SCAN, K);
            }
        }
        __syncthreads();
        const unsigned long long excl = s_excl;
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            const int64_t idx = base + (int64_t)j * kScanThreads + tid;
            if (idx >= a.n_rows) continue;
            const unsigned long long off = excl + local[j];
            a.offsets[idx] = off > 0xffffffffull ? 0xffffffffu : (uint32_t)off;
            const uint32_t c = a.n_tiles[a.rows[idx]];
            if (c == 0) continue;
            // chunks whose first slot falls inside [off, off + c)
            const unsigned long long lo = (off + kDupChunk - 1) / kDupChunk;
            const unsigned long long hi = (off + c - 1) / kDupChunk;
            for (unsigned long long q = lo; q <= hi && q < (unsigned long long)a.n_chunks_max; ++q)
                a.chunk_row[q] = (uint32_t)idx;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// DuplicateWithKeys: one (tile, row) instance per tile of each row's
// rectangle, rows in depth order, tiles row major; + tile-digit histograms.
// ---------------------------------------------------------------------------

struct DupArgs {
    splat_proj proj;
    const uint32_t* rows;      // depth-sorted rows
    const uint32_t* offsets;
    const uint32_t* chunk_row;
    int64_t n_rows;
    const int64_t* n_instances;
    int64_t capacity;
    uint32_t* keys_out;
    uint32_t* vals_out;
    uint32_t* hist;            // [tile_passes][256]
    int tile_passes;
    uint32_t* zero;            // first tile-pass look-back buffer
    int32_t* status;
    int tile_base[SPLAT_MAX_VIEWS];
    int TX[SPLAT_MAX_VIEWS];
};

__global__ void __launch_bounds__(kDupThreads) k_duplicate(DupArgs a)
{
    __shared__ uint32_t s_off[kDupChunk + 1];
    __shared__ uint32_t s_base[kDupChunk + 1];
    __shared__ uint32_t s_w[kDupChunk + 1];
    __shared__ uint32_t s_tx[kDupChunk + 1];
    __shared__ uint32_t s_row[kDupChunk + 1];
    __shared__ uint32_t s_hist[4][kRadix];
    if (status_failed(a.status)) return;
    const int64_t K = min(*a.n_instances, a.capacity);
    const int tid = threadIdx.x;
    for (int i = tid; i < 4 * kRadix; i += kDupThreads) (&s_hist[0][0])[i] = 0;
    {
        const int64_t nz = ((K + kSortPart - 1) / kSortPart) * kRadix;
        for (int64_t i = blockIdx.x * (int64_t)kDupThreads + tid; i < nz; i += (int64_t)gridDim.x * kDupThreads)
            a.zero[i] = 0;
    }
    const int64_t chunks = (K + kDupChunk - 1) / kDupChunk;
    const int64_t N = a.proj.n;
    __syncthreads();
    for (int64_t c = blockIdx.x; c < chunks; c += gridDim.x) {
        const int64_t s0 = c * kDupChunk;
        const int64_t s1 = min(s0 + kDupChunk, K);
        const int64_t j0 = a.chunk_row[c];
        int64_t j1 = (c + 1 < chunks) ? (int64_t)a.chunk_row[c + 1] : j0 + (s1 - s0) - 1;
        j1 = min(j1, a.n_rows - 1);
        j1 = min(j1, j0 + kDupChunk);  // a chunk spans at most kDupChunk + 1 rows
        const int cnt = (int)(j1 - j0 + 1);
        for (int q = tid; q < cnt; q += kDupThreads) {
            const int64_t j = j0 + q;
            const uint32_t row = a.rows[j];
            const int v = (int)(row / N);
            const int4 rc = ((const int4*)a.proj.rect)[row];
            s_off[q] = a.offsets[j];
            s_base[q] = (uint32_t)(a.tile_base[v] + rc.y * a.TX[v] + rc.x);
            s_w[q] = (uint32_t)max(rc.z - rc.x, 1);
            s_tx[q] = (uint32_t)a.TX[v];
            s_row[q] = row;
        }
        __syncthreads();
        for (int64_t s = s0 + tid; s < s1; s += kDupThreads) {
            // last q with s_off[q] <= s
            int lo = 0, hi = cnt - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if ((int64_t)s_off[mid] <= s) lo = mid; else hi = mid - 1;
            }
            const uint32_t l = (uint32_t)(s - s_off[lo]);
            const uint32_t w = s_w[lo];
            const uint32_t ty = l / w, tx = l - ty * w;
            const uint32_t key = s_base[lo] + ty * s_tx[lo] + tx;
            a.keys_out[s] = key;
            a.vals_out[s] = s_row[lo];
            for (int p = 0; p < a.tile_passes; ++p) atomicAdd(&s_hist[p][(key >> (8 * p)) & 0xff], 1u);
        }
        __syncthreads();
    }
    for (int i = tid; i < a.tile_passes * kRadix; i += kDupThreads) {
        const uint32_t h = (&s_hist[0][0])[i];
        if (h) atomicAdd(&a.hist[i], h);
    }
}

// IdentifyTileRanges: [start, end) of each tile's run in the sorted keys.
__global__ void __launch_bounds__(256) k_ranges(const uint32_t* keys, const int64_t* n_instances, int64_t capacity,
                                                uint2* ranges, int32_t* status)
{
    if (status_failed(status)) return;
    const int64_t K = min(*n_instances, capacity);
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < K; s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = keys[s];
        if (s == 0 || keys[s - 1] != k) ranges[k].x = (uint32_t)s;
        if (s == K - 1 || keys[s + 1] != k) ranges[k].y = (uint32_t)(s + 1);
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

struct SortLayout {
    int64_t n_rows, capacity;
    int64_t parts_d, parts_t, parts_scan, n_chunks;
    size_t off_dkeys[2], off_dvals[2], off_offsets, off_chunk, off_scan_lb, off_dlb[2], off_tlb[2], off_tkeys,
        off_tvals, off_hist, off_tickets;
    size_t bytes;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

SortLayout sort_layout(int64_t n_rows, int64_t capacity)
{
    SortLayout L{};
    L.n_rows = n_rows;
    L.capacity = capacity;
    L.parts_d = (n_rows + kSortPart - 1) / kSortPart;
    L.parts_t = (capacity + kSortPart - 1) / kSortPart;
    L.parts_scan = (n_rows + kScanPart - 1) / kScanPart;
    L.n_chunks = (capacity + kDupChunk - 1) / kDupChunk + 1;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align256(o + bytes); return r; };
    for (int b = 0; b < 2; ++b) L.off_dkeys[b] = take(4 * (size_t)n_rows);
    for (int b = 0; b < 2; ++b) L.off_dvals[b] = take(4 * (size_t)n_rows);
    L.off_offsets = take(4 * (size_t)n_rows);
    L.off_chunk = take(4 * (size_t)L.n_chunks);
    L.off_scan_lb = take(8 * (size_t)std::max<int64_t>(L.parts_scan, 1));
    for (int b = 0; b < 2; ++b) L.off_dlb[b] = take(4 * (size_t)kRadix * std::max<int64_t>(L.parts_d, 1));
    for (int b = 0; b < 2; ++b) L.off_tlb[b] = take(4 * (size_t)kRadix * std::max<int64_t>(L.parts_t, 1));
    L.off_tkeys = take(4 * (size_t)capacity);
    L.off_tvals = take(4 * (size_t)capacity);
    L.off_hist = take(4 * (size_t)kRadix * 8);
    L.off_tickets = take(4 * 16);
    L.bytes = o;
    return L;
}

static int sort_ctas_per_sm()
{
    static int cached = 0;
    if (!cached) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_onesweep, kSortThreads, 0) != cudaSuccess || n < 1) n = 1;
        cached = n;
    }
    return cached;
}

cudaError_t launch_bin_sort(const splat_proj& proj, const ViewBatch& vb, const splat_bins& bins, int32_t* status,
                            void* ws, const LaunchCtx& ctx)
{
    const int64_t n_rows = proj.n * vb.V;
    const SortLayout L = sort_layout(n_rows, bins.capacity);
    char* w = (char*)ws;
    auto U = [&](size_t off) { return (uint32_t*)(w + off); };
    cudaStream_t s = ctx.stream;
    cudaError_t err;
    // tickets + histograms, then all tile ranges
    if ((err = cudaMemsetAsync(w + L.off_hist, 0, (L.off_tickets - L.off_hist) + 64, s)) != cudaSuccess) return err;
    if ((err = cudaMemsetAsync(bins.ranges, 0, sizeof(uint32_t) * 2 * (size_t)vb.total_tiles, s)) != cudaSuccess)
        return err;
    if ((err = cudaMemsetAsync(bins.n_instances, 0, sizeof(int64_t), s)) != cudaSuccess) return err;
    if (n_rows == 0) return cudaSuccess;
    uint32_t* hist = U(L.off_hist);
    uint32_t* tickets = U(L.off_tickets);
    const int resident = ctx.num_sms * sort_ctas_per_sm();

    // 1. depth keys + digit histograms; zero the first depth look-back buffer and the scan look-back
    {
        const int blocks = (int)std::min<int64_t>((n_rows + 255) / 256, (int64_t)ctx.num_sms * 8);
        count_launch();
        k_depth_keys<<<blocks, 256, 0, s>>>(proj, n_rows, U(L.off_dkeys[0]), U(L.off_dvals[0]), hist,
                                            U(L.off_dlb[0]), L.parts_d * kRadix,
                                            (unsigned long long*)(w + L.off_scan_lb), L.parts_scan);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    // 2. four depth passes: buffers 0 -> 1 -> 0 -> 1 -> 0
    for (int p = 0; p < 4; ++p) {
        PassArgs a{};
        a.keys_in = U(L.off_dkeys[p & 1]);
        a.vals_in = U(L.off_dvals[p & 1]);
        a.keys_out = p < 3 ? U(L.off_dkeys[(p + 1) & 1]) : nullptr;
        a.vals_out = U(L.off_dvals[(p + 1) & 1]);
        a.n_dev = nullptr;
        a.n_host = n_rows;
        a.cap = n_rows;
        a.hist = hist + p * kRadix;
        a.lb = U(L.off_dlb[p & 1]);
        a.lb_next = p < 3 ? U(L.off_dlb[(p + 1) & 1]) : nullptr;
        a.ticket = tickets + p;
        a.status = status;
        a.stage = SPLAT_STAGE_DEPTH_SORT;
        a.shift = 8 * p;
        a.spin_limit = ctx.spin_limit;
        const int blocks = (int)std::min<int64_t>(L.parts_d, resident);
        count_launch();
        k_onesweep<<<blocks, kSortThreads, 0, s>>>(a);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    const uint32_t* rows = U(L.off_dvals[0]);
    // 3. scan of tile counts in depth order
    {
        ScanArgs a{};
        a.rows = rows;
        a.n_tiles = proj.n_tiles;
        a.n_rows = n_rows;
        a.offsets = U(L.off_offsets);
        a.chunk_row = U(L.off_chunk);
        a.n_chunks_max = L.n_chunks;
        a.lb = (unsigned long long*)(w + L.off_scan_lb);
        a.ticket = tickets + 4;
        a.n_instances = bins.n_instances;
        a.capacity = bins.capacity;
        a.status = status;
        a.spin_limit = ctx.spin_limit;
        const int blocks = (int)std::min<int64_t>(L.parts_scan, (int64_t)ctx.num_sms * 4);
        count_launch();
        k_scan_tiles<<<blocks, kScanThreads, 0, s>>>(a);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    // 4. duplicate
    int bits = 1;
    while ((1ll << bits) < (int64_t)vb.total_tiles) ++bits;
    const int tile_passes = (bits + 7) / 8;
    uint32_t* tk[2] = {U(L.off_tkeys), bins.keys};
    uint32_t* tv[2] = {U(L.off_tvals), bins.vals};
    // the last pass must land in bins: start in the workspace when the pass count is odd
    int cur = (tile_passes & 1) ? 0 : 1;
    {
        DupArgs a{};
        a.proj = proj;
        a.rows = rows;
        a.offsets = U(L.off_offsets);
        a.chunk_row = U(L.off_chunk);
        a.n_rows = n_rows;
        a.n_instances = bins.n_instances;
        a.capacity = bins.capacity;
        a.keys_out = tk[cur];
        a.vals_out = tv[cur];
        a.hist = hist + 4 * kRadix;
        a.tile_passes = tile_passes;
        a.zero = U(L.off_tlb[0]);
        a.status = status;
        for (int v = 0; v < vb.V; ++v) {
            a.tile_base[v] = vb.v[v].tile_base;
            a.TX[v] = vb.v[v].TX;
        }
        const int blocks = ctx.num_sms * 4;
        count_launch();
        k_duplicate<<<blocks, kDupThreads, 0, s>>>(a);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    // 5. tile passes
    for (int p = 0; p < tile_passes; ++p) {
        PassArgs a{};
        a.keys_in = tk[cur];
        a.vals_in = tv[cur];
        a.keys_out = tk[cur ^ 1];
        a.vals_out = tv[cur ^ 1];
        a.n_dev = bins.n_instances;
        a.n_host = 0;
        a.cap = bins.capacity;
        a.hist = hist + (4 + p) * kRadix;
        a.lb = U(L.off_tlb[p & 1]);
        a.lb_next = p + 1 < tile_passes ? U(L.off_tlb[(p + 1) & 1]) : nullptr;
        a.ticket = tickets + 5 + p;
        a.status = status;
        a.stage = SPLAT_STAGE_TILE_SORT;
        a.shift = 8 * p;
        a.spin_limit = ctx.spin_limit;
        const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(L.parts_t, resident));
        count_launch();
        k_onesweep<<<blocks, kSortThreads, 0, s>>>(a);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        cur ^= 1;
    }
    // 6. ranges
    {
        const int blocks = ctx.num_sms * 8;
        count_launch();
        k_ranges<<<blocks, 256, 0, s>>>(bins.keys, bins.n_instances, bins.capacity, (uint2*)bins.ranges, status);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    return cudaSuccess;
}

size_t bin_sort_workspace(int64_t n_rows, int64_t capacity) { return sort_layout(n_rows, capacity).bytes; }

}  // namespace splat
