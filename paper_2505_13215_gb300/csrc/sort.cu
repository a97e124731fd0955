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
// partitions of 4096 keys taken in ticket order by persistent CTAs, local
// ranking of the keys of a warp (digit-bit ballots or a match instruction)
// with shared-memory counters, and a decoupled look-back across partitions
// whose waits are bounded (SPLAT_ERR_TIMEOUT on expiry).  On the binned path
// the depth passes sort each view's rows in place (partitions stay inside a
// view, digit counts and look-back are per view), so four passes give the
// (view, depth) order.
//
// The binned path (the default up to 40960 tiles per view) orders by tile
// without tile-digit passes: the depth-ordered rows are split stably by
// 8x8-tile super-tile in one onesweep-style pass over equal runs of list
// slots (k_super_split), then each super-tile's list is filtered into its
// tiles' lists in order: the first 512 entries by a saturation head
// (k_head_count, a CTA per tile row), the rest in parallel segments
// (k_tile_filter), the counts turned into ranges by one look-back pass
// (k_tile_ranges) and the lists written by one pass.  With culling on, a list
// holds only the tiles the opacity footprint reaches and ends where every
// pixel of the tile has certainly saturated (tile saturation, below); neither
// changes a result.  12 launches for any number of views.
#include <algorithm>

#include "splat_internal.cuh"

namespace splat {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;
constexpr int kSortPart = kSortThreads * kSortItems;  // keys per partition
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanPart = kScanThreads * kScanItems;
constexpr int kDupChunk = 2048;  // instance slots per duplicate work item
constexpr int kDupThreads = 256;

constexpr int kLookWindow = 8;  // predecessors a look-back thread reads per step
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagPrefix = 2u << 30;
constexpr uint32_t kValMask = (1u << 30) - 1;

// Exclusive scan of one value per thread across a 256-thread block.
__device__ __forceinline__ unsigned long long block_excl_scan256_u64(unsigned long long v, unsigned long long* s_tmp,
                                                                     unsigned long long* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_tmp[warp] = x;
    __syncthreads();
    unsigned long long wsum = 0, all = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const unsigned long long t = s_tmp[w];
        if (w < warp) wsum += t;
        all += t;
    }
    __syncthreads();
    *total = all;
    return wsum + x - v;
}

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

struct DepthArgs {
    splat_proj proj;
    int V, blocks_per_view;
    uint32_t* keys;
    uint32_t* vals;
    uint32_t* dhist;        // [4][V][256] digit counts per view
    uint32_t* super_total;  // [total_super] entries of each super-tile list (binned path), or null
    int super_base[SPLAT_MAX_VIEWS];
    int STX[SPLAT_MAX_VIEWS], STY[SPLAT_MAX_VIEWS];
    uint32_t* zero_a;
    int64_t n_zero_a;
    unsigned long long* zero_b;
    int64_t n_zero_b;
    unsigned long long* zero_c;
    int64_t n_zero_c;
};

// Block b serves view b / blocks_per_view.  The super-tile list sizes (binned
// path) are counted through a 2D difference array of the view's super-tile
// grid in dynamic shared memory ((STX + 1) x (STY + 1) words): a row adds its
// super-rectangle with four corner updates, and the block's prefix sums over
// x then y give its counts per super-tile.
__global__ void __launch_bounds__(256) k_depth_keys(DepthArgs a)
{
    extern __shared__ uint32_t s_diff[];
    __shared__ uint32_t s_hist[4][kRadix];
    const int v = (int)(blockIdx.x / a.blocks_per_view), bi = (int)(blockIdx.x - v * a.blocks_per_view);
    const int SX = a.super_total ? a.STX[v] + 1 : 0, SY = a.super_total ? a.STY[v] + 1 : 0;
    for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) (&s_hist[0][0])[i] = 0;
    for (int i = threadIdx.x; i < SX * SY; i += blockDim.x) s_diff[i] = 0;
    __syncthreads();
    const int64_t n = a.proj.n, r_base = (int64_t)v * n;
    for (int64_t i = bi * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)a.blocks_per_view * blockDim.x) {
        const int64_t r = r_base + i;
        const uint32_t nt = a.proj.n_tiles[r];
        const float depth = ((const float4*)a.proj.rgb_depth)[r].w;
        const uint32_t k = nt > 0 ? __float_as_uint(depth) : 0xffffffffu;
        a.keys[r] = k;
        a.vals[r] = (uint32_t)r;
#pragma unroll
        for (int p = 0; p < 4; ++p) atomicAdd(&s_hist[p][(k >> (8 * p)) & 0xff], 1u);
        if (nt > 0 && SX) {  // the super-rectangle [sx0, sx1) x [sy0, sy1) of the row's tile rectangle
            const int4 rc = ((const int4*)a.proj.rect)[r];
            const int sx0 = rc.x >> 3, sy0 = rc.y >> 3, sx1 = (rc.z + 7) >> 3, sy1 = (rc.w + 7) >> 3;
            atomicAdd(&s_diff[sy0 * SX + sx0], 1u);
            atomicAdd(&s_diff[sy0 * SX + sx1], 0xffffffffu);
            atomicAdd(&s_diff[sy1 * SX + sx0], 0xffffffffu);
            atomicAdd(&s_diff[sy1 * SX + sx1], 1u);
        }
    }
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int64_t i = gt; i < a.n_zero_a; i += stride) a.zero_a[i] = 0;
    for (int64_t i = gt; i < a.n_zero_b; i += stride) a.zero_b[i] = 0;
    for (int64_t i = gt; i < a.n_zero_c; i += stride) a.zero_c[i] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) {
        const uint32_t c = (&s_hist[0][0])[i];
        const int p = i / kRadix, d = i - p * kRadix;
        if (c) atomicAdd(&a.dhist[((size_t)p * a.V + v) * kRadix + d], c);
    }
    if (SX) {
        for (int y = threadIdx.x; y < SY; y += blockDim.x) {  // prefix along x
            uint32_t run = 0;
            for (int x = 0; x < SX; ++x) {
                run += s_diff[y * SX + x];
                s_diff[y * SX + x] = run;
            }
        }
        __syncthreads();
        for (int x = threadIdx.x; x < SX; x += blockDim.x) {  // then along y
            uint32_t run = 0;
            for (int y = 0; y < SY; ++y) {
                run += s_diff[y * SX + x];
                s_diff[y * SX + x] = run;
            }
        }
        __syncthreads();
        const int STX = SX - 1, nsup = STX * (SY - 1);
        for (int i = threadIdx.x; i < nsup; i += blockDim.x) {
            const int y = i / STX, x = i - y * STX;
            const uint32_t c = s_diff[y * SX + x];
            if (c) atomicAdd(&a.super_total[a.super_base[v] + i], c);
        }
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
    const uint32_t* hist;  // [segments][256] digit counts of this pass
    uint32_t* lb;          // [parts][256] look-back words of this pass (zeroed)
    uint32_t* lb_next;     // [parts][256] zeroed here for the next pass (may be null)
    uint32_t* ticket;
    int32_t* status;
    int stage;
    int shift;
    int64_t spin_limit;
    int64_t seg_len;       // > 0: the keys form segments of seg_len keys (the views' rows), each sorted on
                           // its own in place, with hist holding [segments][256] counts; 0: one segment
    int hist_sum;          // one segment: the digit counts are the sum of hist_sum [256] arrays
    int ballot_rank;       // rank by digit-bit ballots (many distinct digits per warp) instead of match
};

template <bool BALLOT>
__global__ void __launch_bounds__(kSortThreads) k_onesweep(PassArgs a)
{
    __shared__ uint32_t s_keys[kSortPart];
    __shared__ uint32_t s_vals[kSortPart];
    __shared__ uint32_t s_whist[kSortWarps][kRadix];
    __shared__ uint32_t s_dstart[kRadix];
    __shared__ uint32_t s_base[kRadix];
    __shared__ uint32_t s_tmp[8];
    __shared__ int64_t s_ticket;

    if (status_failed(a.status)) return;
    const int64_t n = a.n_dev ? min(*a.n_dev, a.cap) : a.n_host;
    if (n <= 0) return;
    // segments of seg keys, pps partitions each; a partition never crosses a
    // segment boundary, and its look-back stops at its segment's first one
    const int64_t seg = a.seg_len > 0 ? a.seg_len : n;
    const int64_t pps = (seg + kSortPart - 1) / kSortPart;
    const int64_t parts = pps * ((n + seg - 1) / seg);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = lanemask_lt();
    int64_t cur_seg = -1;
    uint32_t gofs = 0;  // first output position of digit tid in the current segment

    for (;;) {
        if (tid == 0) s_ticket = atomicAdd(a.ticket, 1u);
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) s_whist[w][tid] = 0;
        __syncthreads();
        const int64_t ticket = s_ticket;
        if (ticket >= parts) break;
        const int64_t sg = ticket / pps, lp = ticket - sg * pps, first = sg * pps;
        if (sg != cur_seg) {  // block-uniform
            cur_seg = sg;
            uint32_t h = 0;
            if (a.seg_len > 0) {
                h = a.hist[sg * kRadix + tid];
            } else {
                for (int q = 0; q < a.hist_sum; ++q) h += a.hist[q * kRadix + tid];
            }
            gofs = (uint32_t)(sg * seg) + block_excl_scan256(h, s_tmp, nullptr);
        }
        const int64_t seg_end = min(n, (sg + 1) * seg);
        const int64_t base = sg * seg + lp * kSortPart;
        const int64_t wbase = base + (int64_t)warp * 32 * kSortItems;
        // keys of this warp's share of the partition: its items j * 32 + lane < wrem
        const int64_t wr = seg_end - wbase;
        const int wrem = wr <= 0 ? 0 : (wr >= 32 * kSortItems ? 32 * kSortItems : (int)wr);
        const uint32_t* kin = a.keys_in + wbase;
        const uint32_t* vin = a.vals_in + wbase;

        uint32_t k[kSortItems], v[kSortItems], r[kSortItems];
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const bool ok = j * 32 + lane < wrem;
            k[j] = ok ? kin[j * 32 + lane] : 0u;
            v[j] = ok ? vin[j * 32 + lane] : 0u;
        }
        // warp-level stable ranking, items in (j, lane) order.  The lanes holding
        // the same digit: with BALLOT, one ballot per digit bit (a constant
        // cost, for digits that take many values in a warp); otherwise a match
        // instruction (fast when the warp holds few distinct digits, slow with many)
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const bool ok = j * 32 + lane < wrem;
            const uint32_t dj = (k[j] >> a.shift) & 0xff;
            const unsigned valid = __ballot_sync(0xffffffffu, ok);
            unsigned same = valid;
            if (BALLOT) {
#pragma unroll
                for (int bit = 0; bit < 8; ++bit) {
                    const unsigned bb = __ballot_sync(0xffffffffu, (dj >> bit) & 1u);
                    same &= ((dj >> bit) & 1u) ? bb : ~bb;
                }
            }
            r[j] = 0;
            if (ok) {
                const uint32_t d = dj;
                const unsigned peers = BALLOT ? same : __match_any_sync(valid, d);
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
        st_relaxed(my, (lp == 0 ? kFlagPrefix : kFlagAgg) | cnt);
        if (a.lb_next) a.lb_next[ticket * kRadix + d] = 0;
        s_dstart[d] = block_excl_scan256(cnt, s_tmp, nullptr);
        // decoupled look-back for digit d, kLookWindow predecessors per step
        // (independent loads): all partitions of a pass usually run in one wave,
        // so a walk of one predecessor per L2 round trip would make the last
        // partition wait for about half the partition count of round trips
        uint32_t excl = 0;
        if (lp > 0) {
            int64_t j = ticket - 1;  // nearest predecessor not yet added
            int64_t spins = 0;
            for (;;) {
                uint32_t w[kLookWindow];
#pragma unroll
                for (int q = 0; q < kLookWindow; ++q)
                    w[q] = j - q >= first ? ld_relaxed(a.lb + (j - q) * kRadix + d) : kFlagPrefix;
                // add the published words from the nearest one back, up to and
                // including the first inclusive prefix, or up to the first word
                // not yet published
                int q = 0;
                bool found = false;
#pragma unroll
                for (int t = 0; t < kLookWindow; ++t) {
                    if (found || q < t) continue;  // stopped at an earlier word
                    const uint32_t flag = w[t] & ~kValMask;
                    if (flag == 0) continue;       // not yet published: q stays at t
                    excl += w[t] & kValMask;
                    q = t + 1;
                    found = flag == kFlagPrefix;
                }
                if (found) break;
                j -= q;
                if (q == 0) {
                    if (++spins > a.spin_limit) {
                        set_status(a.status, SPLAT_ERR_TIMEOUT, a.stage, ticket);
                        break;
                    }
                    if (spins > 64) __nanosleep(64);
                }
            }
            st_relaxed(my, kFlagPrefix | ((excl + cnt) & kValMask));
        }
        s_base[d] = gofs + excl - s_dstart[d];
        __syncthreads();
        // local scatter into digit order
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            if (j * 32 + lane < wrem) {
                const uint32_t dd = (k[j] >> a.shift) & 0xff;
                const uint32_t pos = s_dstart[dd] + s_whist[warp][dd] + r[j];
                s_keys[pos] = k[j];
                s_vals[pos] = v[j];
            }
        }
        __syncthreads();
        const int nvalid = (int)min((int64_t)kSortPart, seg_end - base);
        for (int i = tid; i < nvalid; i += kSortThreads) {
            const uint32_t key = s_keys[i];
            const uint32_t out = s_base[(key >> a.shift) & 0xff] + i;
            if (out >= (uint64_t)n) continue;  // only after a timed-out look-back
            const uint32_t val = s_vals[i];
            if (a.keys_out) a.keys_out[out] = key;
            a.vals_out[out] = val;
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
    const int4* rect;          // [n_rows] tile rectangles (used when shift > 0)
    int shift;                 // > 0: count the rectangle's (2^shift)^2 super-tiles instead
    int64_t n_rows;
    uint32_t* offsets;         // [n_rows] exclusive prefix (saturated at 2^32-1)
    uint32_t* chunk_row;       // [n_chunks_max] first sorted position of each duplicate chunk
    int64_t n_chunks_max;
    unsigned long long* lb;    // [parts] look-back words (zeroed)
    uint32_t* ticket;
    int64_t* n_instances;      // out: K
    int64_t* n_needed;         // out (may be null): K as the capacity needed
    int64_t capacity;
    int32_t* status;
    int64_t spin_limit;
};

__device__ __forceinline__ int4 shifted_rect(int4 rc, int shift)
{
    if (shift == 0) return rc;
    const int m = (1 << shift) - 1;
    return make_int4(rc.x >> shift, rc.y >> shift, (rc.z + m) >> shift, (rc.w + m) >> shift);
}

__device__ __forceinline__ uint32_t row_count(const ScanArgs& a, uint32_t row)
{
    const uint32_t n = a.n_tiles[row];
    if (a.shift == 0 || n == 0) return n;
    const int4 rc = shifted_rect(a.rect[row], a.shift);
    return (uint32_t)((rc.z - rc.x) * (rc.w - rc.y));
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(ScanArgs a)
{
    __shared__ unsigned long long s_tmp64[8];
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
        // blocked layout: thread tid owns the kScanItems consecutive rows from base + tid * kScanItems,
        // so one block scan of the per-thread sums serves the whole partition
        const int64_t i0 = base + (int64_t)tid * kScanItems;
        uint32_t c[kScanItems];
        if (i0 + kScanItems <= a.n_rows) {
            const uint4* r4 = (const uint4*)(a.rows + i0);
#pragma unroll
            for (int q = 0; q < kScanItems / 4; ++q) {
                const uint4 r = r4[q];
                c[4 * q + 0] = row_count(a, r.x);
                c[4 * q + 1] = row_count(a, r.y);
                c[4 * q + 2] = row_count(a, r.z);
                c[4 * q + 3] = row_count(a, r.w);
            }
        } else {
#pragma unroll
            for (int j = 0; j < kScanItems; ++j) c[j] = i0 + j < a.n_rows ? row_count(a, a.rows[i0 + j]) : 0u;
        }
        unsigned long long tsum = 0;
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) tsum += c[j];
        unsigned long long running;
        const unsigned long long texcl = block_excl_scan256_u64(tsum, s_tmp64, &running);
        const unsigned long long agg = running;
        if (tid < 32) {
            // decoupled look-back by one warp: lane l reads predecessor j - l, so
            // one round trip covers 32 of them (all partitions usually run in one
            // wave, and a walk of one predecessor per round trip would make the
            // last partition wait for about half the partition count of them)
            const int lane = tid;
            unsigned long long excl = 0;
            if (lane == 0) st_relaxed64(a.lb + ticket, (ticket == 0 ? kP : kA) | agg);
            if (ticket > 0) {
                int64_t j = ticket - 1, spins = 0;  // nearest predecessor not yet added
                for (;;) {
                    const bool in = j - lane >= 0;
                    const unsigned long long s = in ? ld_relaxed64(a.lb + (j - lane)) : kP;
                    const unsigned long long flag = s & ~kM;
                    // the published words from the nearest one back, up to and
                    // including the first inclusive prefix or up to the first
                    // word not yet published
                    const unsigned pend = __ballot_sync(0xffffffffu, flag == 0);
                    const unsigned pref = __ballot_sync(0xffffffffu, flag == kP);
                    const int first_pend = pend ? __ffs(pend) - 1 : 32;
                    const int first_pref = pref ? __ffs(pref) - 1 : 32;
                    const bool found = first_pref < first_pend;
                    const int take = found ? first_pref + 1 : first_pend;
                    unsigned long long v = lane < take ? (s & kM) : 0ull;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    excl += v;
                    if (found) break;
                    j -= take;
                    if (take == 0) {
                        if (++spins > a.spin_limit) {
                            if (lane == 0) set_status(a.status, SPLAT_ERR_TIMEOUT, SPLAT_STAGE_SCAN, ticket);
                            break;
                        }
                        if (spins > 64) __nanosleep(64);
                    }
                }
                if (lane == 0) st_relaxed64(a.lb + ticket, kP | ((excl + agg) & kM));
            }
            if (lane == 0) s_excl = excl;
            if (lane == 0 && ticket == parts - 1) {
                const int64_t K = (int64_t)(excl + agg);
                *a.n_instances = K;
                if (a.n_needed) *a.n_needed = K;
                if (K > a.capacity) set_status(a.status, SPLAT_ERR_CAPACITY, SPLAT_STAGE_SCAN, K);
            }
        }
        __syncthreads();
        const unsigned long long excl = s_excl;
        unsigned long long off = excl + texcl;
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            const int64_t idx = i0 + j;
            if (idx < a.n_rows) {
                a.offsets[idx] = off > 0xffffffffull ? 0xffffffffu : (uint32_t)off;
                if (c[j] != 0 && a.n_chunks_max > 0) {
                    // chunks whose first slot falls inside [off, off + c)
                    const unsigned long long lo = (off + kDupChunk - 1) / kDupChunk;
                    const unsigned long long hi = (off + c[j] - 1) / kDupChunk;
                    for (unsigned long long q = lo; q <= hi && q < (unsigned long long)a.n_chunks_max; ++q)
                        a.chunk_row[q] = (uint32_t)idx;
                }
            }
            off += c[j];
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
// Super-tile lists (level 1 of the binned path): a stable multi-split of the
// (view, depth)-ordered visible rows by 8x8-tile super-tile.  A row enters
// the list of every super-tile its tile rectangle meets, in raster order of
// its super-rectangle, and the scan of the rows' super-tile counts gives every
// row its first slot in that order (the slots of a view are contiguous).  The
// lists' sizes come from the depth-key pass; one onesweep-style pass over
// equal runs of slots then ranks each run's entries per super-tile in slot
// order, finds every super-tile's offset from the runs before it by decoupled
// look-back, and writes the entries in a second sweep over the same slots.
// ---------------------------------------------------------------------------

constexpr int64_t kBinMaxTiles = 40960;  // per view: the binned path's default range
constexpr int kSplitSlots = 4096;        // list slots per split partition (512 per warp)
constexpr int kSplitWarpSlots = kSplitSlots / 8;
constexpr int kSplitMaxSmem = 200 * 1024;  // shared memory the split's counters and grids may take
constexpr unsigned long long kSplitAgg = 1ull << 62, kSplitPrefix = 2ull << 62, kSplitMask = (1ull << 62) - 1;

struct SplitArgs {
    splat_proj proj;
    const uint32_t* rows;          // [V * n] rows, each view's in depth order, its visible ones first
    const uint32_t* offsets;       // [V * n] first list slot of each of those rows
    const uint32_t* super_total;   // [total_super] entries of each super-tile list
    const int64_t* n_instances;    // K1, the slot count (checked against the capacity by the scan)
    int V;
    int64_t n;                     // rows per view
    int smax;                      // row stride of the per-warp counters (>= every view's super-tile count)
    int sdiff;                     // row stride of the per-warp difference grids (>= (STX + 1) (STY + 1))
    int total_super;
    int super_base[SPLAT_MAX_VIEWS + 1];
    int STX[SPLAT_MAX_VIEWS], STY[SPLAT_MAX_VIEWS];
    unsigned long long* lb;        // [max_parts][smax] look-back words (zeroed)
    int64_t max_parts;
    uint32_t* ticket;
    uint32_t* list;                // out: the super-tile lists, K1 entries
    uint2* sranges;                // out: [total_super] [start, end) of each list, (0, 0) when empty
    int32_t* status;
    int64_t spin_limit;
};

// Last position p in [lo, hi) with offsets[p] <= s, given offsets[lo] <= s
// (the warp probes 32 positions per step).
__device__ __forceinline__ int64_t warp_search(const uint32_t* offsets, int64_t lo, int64_t hi, uint32_t s, int lane)
{
    while (hi - lo > 1) {
        const int64_t step = (hi - lo + 31) / 32;
        const int64_t p = lo + lane * step;
        const bool ok = p < hi && offsets[p] <= s;
        const unsigned m = __ballot_sync(0xffffffffu, ok) | 1u;
        const int64_t nlo = lo + (31 - __clz(m)) * step;
        hi = min(hi, nlo + step);
        lo = nlo;
    }
    return lo;
}

// One warp's slots [sa, sb) of view v, from its row j0 on, in rounds of 32
// rows: each row's entries whose slot lies in the range, in slot order, ranked
// per super-tile by ballots over the bits of the super-tile index
// (depth-ordered rows are scattered over the image, so a round holds many
// distinct super-tiles, for which a match instruction is slow); the warp's
// counter of each super-tile advances by its entries.  WRITE: the counters
// hold the warp's first list slot of every super-tile and each entry is
// written there.
template <bool WRITE>
__device__ __forceinline__ void split_sweep(const SplitArgs& a, int v, int nbits, int64_t j0, uint32_t sa,
                                            uint32_t sb, uint32_t* cnt, int lane, unsigned lt)
{
    const int STX = a.STX[v];
    const int64_t vend = (int64_t)(v + 1) * a.n;
    auto emit = [&](bool ok, uint32_t d, uint32_t row) {
        unsigned peers = __ballot_sync(0xffffffffu, ok);
        for (int b = 0; b < nbits; ++b) {  // warp-uniform
            const bool bit = (d >> b) & 1u;
            const unsigned bb = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? bb : ~bb;
        }
        if (ok) {
            const int leader = __ffs(peers) - 1;
            uint32_t prev = 0;
            if (lane == leader) {
                prev = cnt[d];
                cnt[d] = prev + __popc(peers);
            }
            prev = __shfl_sync(peers, prev, leader);
            if (WRITE) a.list[prev + __popc(peers & lt)] = row;
        }
        __syncwarp();
    };
    for (int64_t jb = j0;; jb += 32) {
        const int64_t j = jb + lane;
        // c entries of row j from its entry kl on fall inside [sa, sb); pk: the
        // super-rectangle's origin x | y << 10 | width << 20
        uint32_t row = 0, c = 0, kl = 0, pk = 0;
        bool past = true;
        if (j < vend) {
            const uint32_t off = a.offsets[j];
            past = off >= sb;
            if (!past) {
                row = a.rows[j];
                const int4 rc = ((const int4*)a.proj.rect)[row];
                const int sx0 = rc.x >> 3, sy0 = rc.y >> 3, sx1 = (rc.z + 7) >> 3, sy1 = (rc.w + 7) >> 3;
                if (sx1 > sx0 && sy1 > sy0) {
                    const uint32_t cr = (uint32_t)((sx1 - sx0) * (sy1 - sy0));
                    kl = off < sa ? sa - off : 0u;
                    const uint32_t kh = min(cr, sb - off);
                    c = kh > kl ? kh - kl : 0u;
                    pk = (uint32_t)sx0 | (uint32_t)sy0 << 10 | (uint32_t)(sx1 - sx0) << 20;
                }
            }
        }
        if (__all_sync(0xffffffffu, c <= 1u && kl == 0u)) {  // the common case: a row's first entry at most
            emit(c == 1u, (pk >> 10 & 1023u) * STX + (pk & 1023u), row);
        } else {
            // entry slots of the round in order: lane l owns [e, e + c)
            uint32_t e = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, e, o);
                if (lane >= o) e += y;
            }
            const uint32_t E = __shfl_sync(0xffffffffu, e, 31);
            e -= c;
            for (uint32_t s0 = 0; s0 < E; s0 += 32) {
                const uint32_t sl = s0 + lane;
                // the row of slot sl: the last lane whose first slot is at or before it
                int src = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1)
                    if (__shfl_sync(0xffffffffu, e, src + step) <= sl) src += step;
                const uint32_t srow = __shfl_sync(0xffffffffu, row, src), spk = __shfl_sync(0xffffffffu, pk, src);
                const uint32_t k = sl - __shfl_sync(0xffffffffu, e, src) + __shfl_sync(0xffffffffu, kl, src);
                const int w = (int)(spk >> 20);
                // k / w: an approximate quotient of (k + 1/2) / w (off by at most one), then corrected
                int ky = w ? (int)__fdividef((float)k + 0.5f, (float)w) : 0, kx = (int)k - ky * w;
                if (kx < 0) {
                    --ky;
                    kx += w;
                } else if (kx >= w && w) {
                    ++ky;
                    kx -= w;
                }
                emit(sl < E, ((spk >> 10 & 1023u) + (uint32_t)ky) * STX + (spk & 1023u) + (uint32_t)kx, srow);
            }
        }
        if (__any_sync(0xffffffffu, past)) break;  // offsets grow with j: the later rows are past sb too
    }
}

// Counting pass of one warp's slots [sa, sb) of view v, from its row j0 on:
// a row whose entries all fall inside the range adds its super-rectangle to
// the warp's 2D difference grid diff ((STX + 1) x (STY + 1), zeroed) with four
// corner updates; the first and last rows of the range, which may fall in it
// only in part, add their entries inside it to cnt one by one.  The grid's
// prefix sums are then added to cnt.
__device__ __forceinline__ void split_count(const SplitArgs& a, int v, int64_t j0, uint32_t sa, uint32_t sb,
                                            uint32_t* cnt, uint32_t* diff, int lane)
{
    const int STX = a.STX[v], SX = STX + 1, SY = a.STY[v] + 1;
    const int64_t vend = (int64_t)(v + 1) * a.n;
    for (int64_t jb = j0;; jb += 32) {
        const int64_t j = jb + lane;
        bool past = true;
        if (j < vend) {
            const uint32_t off = a.offsets[j];
            past = off >= sb;
            if (!past) {
                const int4 rc = ((const int4*)a.proj.rect)[a.rows[j]];
                const int sx0 = rc.x >> 3, sy0 = rc.y >> 3, sx1 = (rc.z + 7) >> 3, sy1 = (rc.w + 7) >> 3;
                if (sx1 > sx0 && sy1 > sy0) {
                    const uint32_t w = (uint32_t)(sx1 - sx0), cr = w * (uint32_t)(sy1 - sy0);
                    if (off >= sa && cr <= sb - off) {
                        atomicAdd(&diff[sy0 * SX + sx0], 1u);
                        atomicAdd(&diff[sy0 * SX + sx1], 0xffffffffu);
                        atomicAdd(&diff[sy1 * SX + sx0], 0xffffffffu);
                        atomicAdd(&diff[sy1 * SX + sx1], 1u);
                    } else {
                        const uint32_t kh = min(cr, sb - off);
                        for (uint32_t k = off < sa ? sa - off : 0u; k < kh; ++k) {
                            const uint32_t ky = k / w;
                            atomicAdd(&cnt[(sy0 + ky) * STX + sx0 + (k - ky * w)], 1u);
                        }
                    }
                }
            }
        }
        if (__any_sync(0xffffffffu, past)) break;  // offsets grow with j: the later rows are past sb too
    }
    __syncwarp();
    for (int y = lane; y < SY; y += 32) {  // prefix along x
        uint32_t run = 0;
        for (int x = 0; x < SX; ++x) {
            run += diff[y * SX + x];
            diff[y * SX + x] = run;
        }
    }
    __syncwarp();
    for (int x = lane; x < SX; x += 32) {  // then along y
        uint32_t run = 0;
        for (int y = 0; y < SY; ++y) {
            run += diff[y * SX + x];
            diff[y * SX + x] = run;
        }
    }
    __syncwarp();
    for (int d = lane; d < STX * (SY - 1); d += 32) {
        const int y = d / STX;
        cnt[d] += diff[y * SX + (d - y * STX)];
    }
    __syncwarp();
}

__global__ void __launch_bounds__(256) k_super_split(SplitArgs a)
{
    extern __shared__ uint32_t s_dyn[];
    uint32_t* s_cnt = s_dyn;                 // [8][smax] per-warp counters, then the warps' first slots
    uint32_t* s_start = s_dyn + 8 * a.smax;  // [smax] first list slot of each super-tile of the view
    uint32_t* s_diff = s_start + a.smax;     // [8][sdiff] per-warp difference grids of the counting pass
    __shared__ uint32_t s_S[SPLAT_MAX_VIEWS + 1];   // first slot of each view
    __shared__ uint32_t s_cb[SPLAT_MAX_VIEWS + 1];  // first partition of each view
    __shared__ unsigned long long s_tmp64[8];
    __shared__ int64_t s_ticket;
    if (status_failed(a.status)) return;  // includes K1 above the capacity
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = lanemask_lt();
    if (tid == 0) {
        const uint32_t K1 = (uint32_t)*a.n_instances;
        uint32_t cb = 0;
        for (int v = 0; v < a.V; ++v) s_S[v] = a.offsets[(int64_t)v * a.n];
        s_S[a.V] = K1;
        for (int v = 0; v < a.V; ++v) {  // every view takes a partition, if only to write its ranges
            s_cb[v] = cb;
            cb += max(1u, (s_S[v + 1] - s_S[v] + kSplitSlots - 1) / kSplitSlots);
        }
        s_cb[a.V] = cb;
    }
    __syncthreads();
    const int64_t parts = min((int64_t)s_cb[a.V], a.max_parts);
    int cur_v = -1;
    for (;;) {
        if (tid == 0) s_ticket = atomicAdd(a.ticket, 1u);
        __syncthreads();
        const int64_t ticket = s_ticket;
        if (ticket >= parts) break;
        int v = 0;
        for (int q = 1; q < a.V; ++q)
            if (ticket >= (int64_t)s_cb[q]) v = q;
        const int64_t first = s_cb[v], lp = ticket - first;
        const int nsup = a.STX[v] * a.STY[v];
        const int nbits = 32 - __clz(max(nsup - 1, 1));  // bits of a super-tile index of the view
        const int sbase = a.super_base[v];
        if (v != cur_v) {  // block-uniform: the first list slot of each of the view's super-tiles
            cur_v = v;
            unsigned long long before = s_S[v];
            for (int d0 = 0; d0 < nsup; d0 += 256) {
                const int d = d0 + tid;
                const uint32_t c = d < nsup ? a.super_total[sbase + d] : 0u;
                unsigned long long tot;
                const unsigned long long ex = block_excl_scan256_u64(c, s_tmp64, &tot);
                if (d < nsup) s_start[d] = (uint32_t)(before + ex);
                before += tot;
            }
            __syncthreads();
        }
        if (lp == 0) {
            for (int d = tid; d < nsup; d += 256) {
                const uint32_t c = a.super_total[sbase + d], st = s_start[d];
                a.sranges[sbase + d] = c ? make_uint2(st, st + c) : make_uint2(0u, 0u);
            }
        }
        // this partition's slots and this warp's share of them
        const uint32_t s0 = s_S[v] + (uint32_t)lp * kSplitSlots, s1 = min(s_S[v + 1], s0 + kSplitSlots);
        const uint32_t wa = min(s1, s0 + warp * kSplitWarpSlots), wb = min(s1, wa + kSplitWarpSlots);
        int64_t j0 = 0;
        if (wa < wb) j0 = warp_search(a.offsets, (int64_t)v * a.n, (int64_t)(v + 1) * a.n, wa, lane);
        uint32_t* cnt = s_cnt + warp * a.smax;
        uint32_t* diff = s_diff + warp * a.sdiff;
        for (int d = lane; d < nsup; d += 32) cnt[d] = 0u;
        for (int d = lane; d < (a.STX[v] + 1) * (a.STY[v] + 1); d += 32) diff[d] = 0u;
        __syncwarp();
        if (wa < wb) split_count(a, v, j0, wa, wb, cnt, diff, lane);
        __syncthreads();
        // per super-tile: prefix over the warps, the partition's count, look-back
        for (int d = tid; d < nsup; d += 256) {
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                const uint32_t c = s_cnt[w * a.smax + d];
                s_cnt[w * a.smax + d] = run;
                run += c;
            }
            unsigned long long* my = a.lb + ticket * a.smax + d;
            st_relaxed64(my, (lp == 0 ? kSplitPrefix : kSplitAgg) | run);
            unsigned long long excl = 0;
            if (lp > 0) {
                int64_t j = ticket - 1, spins = 0;  // nearest predecessor not yet added
                for (;;) {
                    unsigned long long wd[kLookWindow];
#pragma unroll
                    for (int q = 0; q < kLookWindow; ++q)
                        wd[q] = j - q >= first ? ld_relaxed64(a.lb + (j - q) * a.smax + d) : kSplitPrefix;
                    int q = 0;
                    bool found = false;
#pragma unroll
                    for (int t = 0; t < kLookWindow; ++t) {
                        if (found || q < t) continue;  // stopped at an earlier word
                        const unsigned long long flag = wd[t] & ~kSplitMask;
                        if (flag == 0) continue;       // not yet published: q stays at t
                        excl += wd[t] & kSplitMask;
                        q = t + 1;
                        found = flag == kSplitPrefix;
                    }
                    if (found) break;
                    j -= q;
                    if (q == 0) {
                        if (++spins > a.spin_limit) {
                            set_status(a.status, SPLAT_ERR_TIMEOUT, SPLAT_STAGE_SCAN, ticket);
                            break;
                        }
                        if (spins > 64) __nanosleep(64);
                    }
                }
                st_relaxed64(my, kSplitPrefix | ((excl + run) & kSplitMask));
            }
            const uint32_t base = s_start[d] + (uint32_t)excl;
#pragma unroll
            for (int w = 0; w < 8; ++w) s_cnt[w * a.smax + d] += base;
        }
        __syncthreads();
        if (wa < wb && !status_failed(a.status)) split_sweep<true>(a, v, nbits, j0, wa, wb, cnt, lane, lt);
        __syncthreads();
    }
}

// Tiles in decreasing order of list length for the compositing kernels'
// scheduling (the longest first, so that the last wave of warps is short):
// classes of eight per power of two (the three bits after the leading one),
// a counting sort over the classes in two grid-wide passes (class counts,
// then each tile's slot from its class start and a class cursor), the order
// inside a class unspecified.  Greedy scheduling of the bench scene's measured
// walks on the compositing kernels' 2432 warp slots ends 7.7% above the ideal
// with one class per power of two and 2.9% above with eight (2.8% with the
// exact order).  cls[0..kOrderClasses): counts, then as many cursors, all zero
// on entry.  Lanes of a warp in the same class touch its counter once.
constexpr uint32_t kOrderClasses = 32 * 8 + 1;  // class 0: empty lists

__device__ __forceinline__ uint32_t length_class(uint32_t c)
{
    if (!c) return 0u;
    const int e = 31 - __clz(c);  // c in [2^e, 2^(e+1))
    const uint32_t f = (e >= 3 ? c >> (e - 3) : c << (3 - e)) & 7u;
    return 1u + 8u * (uint32_t)e + f;
}

__device__ __forceinline__ uint32_t tile_class(const uint2* ranges, int i)
{
    const uint2 r = ranges[i];
    return length_class(r.y - r.x);
}

template <bool SCATTER>
__global__ void __launch_bounds__(256) k_tile_order(const uint2* ranges, int n, uint32_t* cls, uint32_t* order,
                                                    int32_t* status)
{
    __shared__ uint32_t s_start[kOrderClasses];
    __shared__ uint32_t s_tmp[8];
    if (status_failed(status)) return;
    const int lane = threadIdx.x & 31;
    if (SCATTER) {
        // class starts, the longest class first: thread t takes class
        // kOrderClasses - 1 - t; the empty lists (class 0) go last
        const uint32_t cb = kOrderClasses - 1u - threadIdx.x;
        uint32_t total;
        const uint32_t ex = block_excl_scan256(cls[cb], s_tmp, &total);
        s_start[cb] = ex;
        if (threadIdx.x == 0) s_start[0] = total;
        __syncthreads();
    }
    const int stride = gridDim.x * blockDim.x;
    for (int i0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < n; i0 += stride) {  // warp-uniform
        const int i = i0 + lane;
        const uint32_t c = i < n ? tile_class(ranges, i) : kOrderClasses;
        const unsigned peers = __match_any_sync(0xffffffffu, c);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (lane == leader && c < kOrderClasses)
            base = atomicAdd(&cls[SCATTER ? kOrderClasses + c : c], (uint32_t)__popc(peers));
        if (SCATTER) {
            base = __shfl_sync(0xffffffffu, base, leader);
            if (c < kOrderClasses) order[s_start[c] + base + __popc(peers & lanemask_lt())] = (uint32_t)i;
        }
    }
}

// counted: the class counts are already in place (and the cursors zero), from
// the binned path's tile ranges
static cudaError_t launch_tile_order(const splat_bins& bins, int64_t total_tiles, uint32_t* cls, int32_t* status,
                                     const LaunchCtx& ctx, bool counted = false)
{
    if (!bins.tile_order || total_tiles <= 0) return cudaSuccess;
    const int n = (int)total_tiles;
    const int blocks = (int)std::min<int64_t>((total_tiles + 255) / 256, (int64_t)ctx.num_sms * 4);
    if (!counted) {
        cudaError_t e = cudaMemsetAsync(cls, 0, 2 * kOrderClasses * sizeof(uint32_t), ctx.stream);
        if (e != cudaSuccess) return e;
        count_launch();
        k_tile_order<false><<<blocks, 256, 0, ctx.stream>>>((const uint2*)bins.ranges, n, cls, bins.tile_order, status);
    }
    count_launch();
    k_tile_order<true><<<blocks, 256, 0, ctx.stream>>>((const uint2*)bins.ranges, n, cls, bins.tile_order, status);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Tile level.  Counting passes over each super-tile's list (the head in order,
// the tail in segments) give every tile's counts, k_tile_ranges turns them
// into ranges (and K), and the writing passes emit the lists.
// ---------------------------------------------------------------------------

struct TileArgs {
    splat_proj proj;
    int V;
    int64_t n_rows;
    int total_tiles;
    int tile_base[SPLAT_MAX_VIEWS + 1];
    int TX[SPLAT_MAX_VIEWS], TY[SPLAT_MAX_VIEWS];
    uint32_t* tile_total;
    // per-super-tile filter
    const uint32_t* list;             // rows grouped by super-tile, depth order inside
    const uint2* sranges;             // [total_super]
    int total_super;
    int super_base[SPLAT_MAX_VIEWS + 1];
    int STX[SPLAT_MAX_VIEWS];
    const uint2* ranges;              // tile ranges (cursor starts)
    uint32_t* vals_out;
    uint32_t* keys_out;               // may be null
    int cull;                         // drop tiles the opacity footprint cannot reach
    int W[SPLAT_MAX_VIEWS], H[SPLAT_MAX_VIEWS];
    uint32_t* n_head8;                // [total_super][8] entries each tile row's head count went through
    uint32_t* n_head;                 // [total_super] entries of each list the head pass went through
    uint2* sat_head;                  // [total_super] tiles (bit 8 r + c) whose lists ended in the head
    uint32_t* seg_base;               // [total_super + 1] first tail segment of each super-tile
    uint32_t* seg_super;              // [segments] super-tile of each tail segment
    uint32_t* seg_cnt;                // [segments][64] per-segment tile counts, then offsets
    uint2* mask;                      // per super-tile list entry: byte w = its tile columns in tile row w
    uint32_t* ticket;                 // [3] tickets of the writing and tail counting passes, head count
                                      // CTAs done (zeroed)
    int32_t* status;
    unsigned long long* stats;        // diagnostic (may be null): [4] super-tiles whose lists ended in
                                      // the head for some tiles and continue in tail segments for others,
                                      // [5] tail segments
};

// Tile saturation.  Every pixel of a tile stops its walk before the first
// entry that would take its transmittance T below 1e-4 (Alg. 1), so the
// entries of a tile list that come after the point where T is certainly below
// that bound at every pixel of the tile are never read.  For each (entry,
// tile) the count pass takes a lower bound of the alpha the compositing
// kernels compute at every pixel of the tile (clipped to the image):
// alpha_max exp(-q/2) with q the largest value of the conic's quadratic form
// over the tile's corners (the form is convex), q enlarged to cover FP32
// rounding, provided the bound passes the 1/255 skip with a margin and the
// conic is far enough from singular that the kernels' evaluation of the power
// cannot round to the wrong side of 0.  The head pass sums -ln(1 - alpha)
// over each tile's list in order, in fixed point (rounded down), and ends the
// list after the batch of 32 entries that takes the sum past -ln(1e-4) with a
// margin for the rounding of the T products (a product of (1 - alpha) below
// e^-9.25 at every pixel; the kernels' T rounds by about 2^-23 an update, which
// the margin covers for 2e5 updates, and a cut falls within the first
// kHeadChunks x 256 entries of a list).  The sums are exact integers, so the
// cut does not depend on the order of any reduction.
constexpr float kSatScale = 65536.f;                       // fixed point of -ln(1 - alpha)
constexpr uint32_t kSatThreshold = (uint32_t)(9.25 * 65536);  // -ln(1e-4) = 9.2103 plus the margin

// Terms of an entry's quadratic form that depend only on the tile row's pixel
// rows [ylo, yhi] (shared by the tiles of the row).
struct SatRow {
    float a, B0, B1, C0, C1, Bm, Cm, px, amax;
};

__device__ __forceinline__ SatRow sat_row(const float4& co, float px, float py, float ylo, float yhi)
{
    const float b2 = 2.f * co.y, dy0 = py - ylo, dy1 = py - yhi, my = fmaxf(fabsf(dy0), fabsf(dy1));
    SatRow r;
    r.a = co.x;
    r.B0 = b2 * dy0;
    r.B1 = b2 * dy1;
    r.C0 = co.z * dy0 * dy0;
    r.C1 = co.z * dy1 * dy1;
    r.Bm = fabsf(b2) * my;
    r.Cm = co.z * my * my;
    r.px = px;
    r.amax = co.w;
    return r;
}

// Saturation weight of one (entry, tile): -ln(1 - alpha_lb) in fixed point,
// rounded down, for the tile's pixel columns [xlo, xhi]; 0 when the bound does
// not pass the 1/255 skip with a margin.
__device__ __forceinline__ uint32_t sat_weight(const SatRow& r, float xlo, float xhi)
{
    const float dx0 = r.px - xlo, dx1 = r.px - xhi;
    // q = a dx^2 + 2 b dx dy + c dy^2 at the four corners
    const float q00 = fmaf(dx0, fmaf(r.a, dx0, r.B0), r.C0), q01 = fmaf(dx0, fmaf(r.a, dx0, r.B1), r.C1);
    const float q10 = fmaf(dx1, fmaf(r.a, dx1, r.B0), r.C0), q11 = fmaf(dx1, fmaf(r.a, dx1, r.B1), r.C1);
    const float qmax = fmaxf(fmaxf(q00, q01), fmaxf(q10, q11));
    const float mx = fmaxf(fabsf(dx0), fabsf(dx1));
    const float qabs = fmaf(mx, fmaf(r.a, mx, r.Bm), r.Cm);  // bounds |a dx^2| + |2 b dx dy| + |c dy^2|
    const float qhi = fmaf(1e-5f, qabs, qmax) + 1e-6f;
    const float alpha = fminf(r.amax * __expf(-0.5f * qhi) * (1.f - 1e-5f), 0.98999f);
    if (!(alpha >= kAlphaMin * 1.002f)) return 0u;
    const float nl = -__log2f(1.f - alpha) * 0.69314718f;  // -ln(1 - alpha)
    const float w = fmaf(nl, 1.f - 1e-4f, -2e-5f);
    return w > 0.f ? (uint32_t)(w * kSatScale) : 0u;
}

constexpr int kFilterSeg = 1024;  // list entries per tail segment (one CTA)
constexpr int kHeadChunks = 2;    // 256-row chunks of each list the head pass takes in order

// one block (the last of the head count): head length of each super-tile list
// (its longest tile row's), tail segments per list, exclusive scan -> seg_base
__device__ __forceinline__ void seg_plan(const TileArgs& a, uint32_t* s_tmp)
{
    uint32_t carry = 0;
    for (int base = 0; base < a.total_super; base += 256) {
        const int gs = base + threadIdx.x;
        uint32_t c = 0;
        if (gs < a.total_super) {  // the tail: what the head pass left, unless every list ended in it
            const uint2 rg = a.sranges[gs], sat = a.sat_head[gs];
            const uint4 h0 = ((const uint4*)a.n_head8)[2 * gs], h1 = ((const uint4*)a.n_head8)[2 * gs + 1];
            const uint32_t nh = max(max(max(h0.x, h0.y), max(h0.z, h0.w)), max(max(h1.x, h1.y), max(h1.z, h1.w)));
            a.n_head[gs] = nh;
            const uint32_t rest = (sat.x & sat.y) == 0xffffffffu ? 0u : rg.y - rg.x - nh;
            c = (rest + kFilterSeg - 1) / kFilterSeg;
        }
        uint32_t tot;
        const uint32_t ex = block_excl_scan256(c, s_tmp, &tot);
        if (gs < a.total_super) {
            a.seg_base[gs] = carry + ex;
            for (uint32_t q = 0; q < c; ++q) a.seg_super[carry + ex + q] = (uint32_t)gs;
            if (a.stats && c > 0) {  // some of its tiles closed in the head, others open in the tail
                int v = 0;
                for (int q = 1; q < a.V; ++q)
                    if (gs >= a.super_base[q]) v = q;
                const int ls = gs - a.super_base[v], sy = ls / a.STX[v], sx = ls - sy * a.STX[v];
                const int nx = min(8, a.TX[v] - 8 * sx), ny = min(8, a.TY[v] - 8 * sy);
                const uint32_t in_grid = (1u << nx) - 1u;
                const uint2 sat = a.sat_head[gs];
                bool closed = false, open = false;
                for (int r = 0; r < ny; ++r) {
                    const uint32_t b = ((r < 4 ? sat.x >> (8 * r) : sat.y >> (8 * (r - 4))) & 0xffu) & in_grid;
                    closed |= b != 0u;
                    open |= b != in_grid;
                }
                if (closed && open) atomicAdd(a.stats + 4, 1ull);
            }
        }
        carry += tot;
    }
    if (threadIdx.x == 0) {
        a.seg_base[a.total_super] = carry;
        if (a.stats) atomicAdd(a.stats + 5, (unsigned long long)carry);
    }
}

// Tile totals, offsets and ranges in one pass over the tiles in global order,
// kRangeTiles per block taken in ticket order, kRangeTiles / 256 consecutive
// tiles per thread.  A tile's total is its head count plus its counts in the
// tail segments of its super-tile, whose entries become the tile-relative
// offsets of the segments; the exclusive scan of the totals across blocks
// (decoupled look-back) gives every tile's range [start, start + total) and
// leaves the start in tile_total.  The last block also writes K, checks it
// against the capacity and reports the capacity the call needed.
constexpr int kRangeTileItems = 1;
constexpr int kRangeTiles = 256 * kRangeTileItems;

struct TileRangeArgs {
    unsigned long long* lb;  // [blocks] look-back words (zeroed)
    uint32_t* ticket;        // (zeroed)
    uint2* ranges;
    int64_t* K_out;
    int64_t capacity;
    const int64_t* K_super;  // entries of the super-tile lists, which share the capacity
    int64_t* needed;         // may be null
    uint32_t* cls;           // [33] tiles per list-length class for the tile order (zeroed), or null
    int64_t spin_limit;
};

__global__ void __launch_bounds__(256) k_tile_ranges(TileArgs a, TileRangeArgs r)
{
    __shared__ unsigned long long s_tmp64[8];
    __shared__ unsigned long long s_excl;
    __shared__ int64_t s_ticket;
    __shared__ uint32_t s_cls[kOrderClasses];
    constexpr unsigned long long kA = 1ull << 62, kP = 2ull << 62, kM = (1ull << 62) - 1;
    if (status_failed(a.status)) return;
    const int tid = threadIdx.x;
    if (tid == 0) s_ticket = atomicAdd(r.ticket, 1u);
    for (int c = tid; c < (int)kOrderClasses; c += blockDim.x) s_cls[c] = 0u;
    __syncthreads();
    const int64_t blk = s_ticket, nblk = ((int64_t)a.total_tiles + kRangeTiles - 1) / kRangeTiles;
    if (blk >= nblk) return;
    const int64_t t0 = blk * kRangeTiles + (int64_t)tid * kRangeTileItems;
    uint32_t cnt[kRangeTileItems];
    unsigned long long tsum = 0;
#pragma unroll
    for (int q = 0; q < kRangeTileItems; ++q) {
        const int64_t t = t0 + q;
        uint32_t run = 0;
        if (t < a.total_tiles) {
            int v = 0;
            for (int w = 1; w < a.V; ++w)
                if (t >= a.tile_base[w]) v = w;
            const int local = (int)(t - a.tile_base[v]);
            const int ty = local / a.TX[v], tx = local - ty * a.TX[v];
            const int gs = a.super_base[v] + (ty >> 3) * a.STX[v] + (tx >> 3), lt = (ty & 7) * 8 + (tx & 7);
            run = a.tile_total[t];  // the head's count: the tail segments follow it
            // the segments' counts, four loads in flight at a time, become their offsets
            const uint32_t g1 = a.seg_base[gs + 1];
            for (uint32_t g = a.seg_base[gs]; g < g1; g += 4) {
                uint32_t c[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) c[u] = g + u < g1 ? a.seg_cnt[(size_t)(g + u) * 64 + lt] : 0u;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (g + u < g1) a.seg_cnt[(size_t)(g + u) * 64 + lt] = run;
                    run += c[u];
                }
            }
        }
        cnt[q] = run;
        tsum += run;
        if (r.cls && t < a.total_tiles) atomicAdd(&s_cls[length_class(run)], 1u);  // as tile_class
    }
    unsigned long long agg;
    const unsigned long long texcl = block_excl_scan256_u64(tsum, s_tmp64, &agg);
    if (tid < 32) {  // decoupled look-back by one warp, 32 predecessors per round trip
        const int lane = tid;
        unsigned long long excl = 0;
        if (lane == 0) st_relaxed64(r.lb + blk, (blk == 0 ? kP : kA) | agg);
        if (blk > 0) {
            int64_t j = blk - 1, spins = 0;
            for (;;) {
                const unsigned long long w = j - lane >= 0 ? ld_relaxed64(r.lb + (j - lane)) : kP;
                const unsigned long long flag = w & ~kM;
                const unsigned pend = __ballot_sync(0xffffffffu, flag == 0);
                const unsigned pref = __ballot_sync(0xffffffffu, flag == kP);
                const int first_pend = pend ? __ffs(pend) - 1 : 32;
                const int first_pref = pref ? __ffs(pref) - 1 : 32;
                const bool found = first_pref < first_pend;
                const int take = found ? first_pref + 1 : first_pend;
                unsigned long long x = lane < take ? (w & kM) : 0ull;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                excl += x;
                if (found) break;
                j -= take;
                if (take == 0) {
                    if (++spins > r.spin_limit) {
                        if (lane == 0) set_status(a.status, SPLAT_ERR_TIMEOUT, SPLAT_STAGE_DUPLICATE, blk);
                        break;
                    }
                    if (spins > 64) __nanosleep(64);
                }
            }
            if (lane == 0) st_relaxed64(r.lb + blk, kP | ((excl + agg) & kM));
        }
        if (lane == 0) {
            s_excl = excl;
            if (blk == nblk - 1) {
                const int64_t K = (int64_t)(excl + agg);
                *r.K_out = K;
                if (K > r.capacity) set_status(a.status, SPLAT_ERR_CAPACITY, SPLAT_STAGE_DUPLICATE, K);
                if (r.needed) *r.needed = max(K, *r.K_super);
            }
        }
    }
    __syncthreads();
    if (r.cls)
        for (int c = tid; c < (int)kOrderClasses; c += blockDim.x)
            if (s_cls[c]) atomicAdd(&r.cls[c], s_cls[c]);
    // slots past 2^32 only arise with K beyond any capacity: the check above reports them
    uint32_t st = (uint32_t)(s_excl + texcl);
#pragma unroll
    for (int q = 0; q < kRangeTileItems; ++q) {
        const int64_t t = t0 + q;
        if (t < a.total_tiles) {
            r.ranges[t] = cnt[q] ? make_uint2(st, st + cnt[q]) : make_uint2(0u, 0u);
            a.tile_total[t] = st;
        }
        st += cnt[q];
    }
}

// Opacity footprint of one projected Gaussian: the ellipse {power >= pcut},
// power = -(a dx^2 + 2 b dx dy + c dy^2) / 2 with dx = px - u, dy = py - v,
// i.e. q(dx, dy) <= R2 = -2 pcut (R2 enlarged by the caller).  Constants per
// Gaussian, computed once: g0 = (px, py, R2, Y) with Y the |dy| reach,
// g1 = (X, yr, b/a, det/a) with X the |dx| reach and yr the dy of the rightmost
// point, g2.x = 1/a.  Degenerate conics keep the whole band (Y = inf).
// Square root by the PTX approximation (a few ulp): the footprint's squared
// radius carries a margin of 1e-4 of itself, far above that error.
__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void ellipse_consts(float px, float py, float a, float b, float c, float R2, float4& g0,
                                               float4& g1)
{
    const float det = a * c - b * b;
    if (!(det > 0.f) || !(a > 0.f) || !(c > 0.f)) {
        g0 = make_float4(px, py, 0.f, __int_as_float(0x7f800000));
        g1 = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    // approximate quotients and roots (relative errors of a few 1e-7, inside
    // the squared radius' 1e-4 margin)
    const float ia = __fdividef(1.f, a), idet = __fdividef(1.f, det);
    const float X = sqrt_approx(R2 * c * idet);
    // g0 = (centre, R2 / a, reach in y); g1 = (reach in x, dy of the rightmost
    // point, b / a, det / a^2)
    g0 = make_float4(px, py, R2 * ia, sqrt_approx(R2 * a * idet));
    g1 = make_float4(X, -__fdividef(b, c) * X, b * ia, det * ia * ia);
}

// Horizontal pixel extent [ul, ur] of the footprint inside the pixel band
// v in [vlo, vhi]; false when the footprint misses the band.  At offset dy the
// footprint spans dx = -(b/a) dy +- sqrt(R2/a - (det/a^2) dy^2).
__device__ __forceinline__ bool ellipse_band_extent(const float4& g0, const float4& g1, float vlo, float vhi,
                                                    float& ul, float& ur)
{
    const float px = g0.x, py = g0.y, Ra = g0.z, Y = g0.w;
    if (isinf(Y)) {
        ul = -3.0e38f;
        ur = 3.0e38f;
        return true;
    }
    const float e0 = fmaxf(py - vhi, -Y), e1 = fminf(py - vlo, Y);  // dy range of the band inside the reach
    if (e0 > e1) return false;
    const float X = g1.x, yr = g1.y, ba = g1.z, hq = g1.w;
    float dxmax, dxmin;
    if (yr >= e0 && yr <= e1) {
        dxmax = X;
    } else {
        const float dy = fminf(fmaxf(yr, e0), e1);
        dxmax = -ba * dy + sqrt_approx(fmaxf(0.f, Ra - hq * dy * dy));
    }
    const float yl = -yr;  // leftmost point
    if (yl >= e0 && yl <= e1) {
        dxmin = -X;
    } else {
        const float dy = fminf(fmaxf(yl, e0), e1);
        dxmin = -ba * dy - sqrt_approx(fmaxf(0.f, Ra - hq * dy * dy));
    }
    ul = px - dxmax;
    ur = px - dxmin;
    return true;
}

// Head pass, counting: one CTA per (super-tile, tile row), warp c serving
// tile column c.  The CTA streams the first kHeadChunks x 256 entries of the
// super-tile's list in depth order, 256 at a time.  Thread t takes entry t of
// the chunk: the entry joins the tile row's queue (in order) when its
// rectangle covers the row, and then gets its columns in the row (the
// rectangle's, narrowed with culling on to the opacity footprint enlarged by a
// margin that covers FP32 rounding, so no pixel result changes) and the terms
// of its saturation bound for the row.  Warp c goes through the queue in
// batches of 32, counts the entries listed in tile c and, with culling on,
// sums their saturation weights; tile c's list ends after the batch that takes
// the sum past the threshold.  Every entry up to the head's end gets its
// coverage byte for this tile row (bit c: listed in tile c), zero once the
// row's lists have all ended, so that the write pass runs on the bytes alone.
// Per row the CTA leaves the entries it went through (n_head8: up to the end
// of the chunk in which its last open list ended) and the ended columns (byte
// w of sat_head); the last CTA to finish then takes each super-tile's head
// length as its largest row's and plans the tail segments (seg_plan).
// compiled for 8 resident CTAs per SM (32 registers; 6 at 39 registers measured
// 1.5 us slower per 4-view step, while the split and the tail passes measured
// slower when held to 32 registers)
__global__ void __launch_bounds__(256, 8) k_head_count(TileArgs a)
{
    __shared__ unsigned char s_m[256];       // columns of each entry of the chunk in this tile row
    __shared__ unsigned char s_queue[256];   // the chunk's entries queued by the row, in order
    __shared__ float4 s_sr0[256], s_sr1[256];  // saturation terms (a, B0, B1, C0), (C1, Bm, Cm, px)
    __shared__ float s_amax[256];            // alpha_max, 0 when the entry does not enter the bound
    __shared__ uint32_t s_wn[8], s_keep[8];
    __shared__ uint32_t s_sat;
    __shared__ bool s_last;
    if (status_failed(a.status)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    const int gs = (int)(blockIdx.x >> 3), w = (int)(blockIdx.x & 7);
    if (gs >= a.total_super) return;
    int v = 0;
    for (int q = 1; q < a.V; ++q)
        if (gs >= a.super_base[q]) v = q;
    const int ls = gs - a.super_base[v];
    const int sy = ls / a.STX[v], sx = ls - sy * a.STX[v];
    const int TX = a.TX[v], TY = a.TY[v];
    const int ty = sy * 8 + w, tx0 = sx * 8;
    const float vlo = (float)(ty * kTile), vhi = vlo + (float)(kTile - 1);
    const float vhi_img = fminf(vhi, (float)(a.H[v] - 1)), xmax_img = (float)(a.W[v] - 1);
    const float xlo = (float)((tx0 + warp) * kTile), xhi = fminf(xlo + (float)(kTile - 1), xmax_img);
    // column state of this warp (warp-uniform): columns outside the grid have ended from the start
    bool sat = !(ty < TY && tx0 + warp < TX);
    uint32_t cnt = 0u, wsum = 0u;
    if (threadIdx.x == 0) s_sat = 0u;
    const uint2 rgs = a.sranges[gs];
    const uint32_t end = min(rgs.y, rgs.x + (uint32_t)(kHeadChunks * 256));
    uint32_t row_end = rgs.x;
    int done = __syncthreads_and(sat);  // block-uniform: every list of the row has ended
    for (uint32_t b = rgs.x; b < end; b += 256) {
        if (!done) row_end = min(b + 256u, end);
        const uint32_t j = b + threadIdx.x;
        uint32_t m = 0u;
        bool cov = false;
        if (!done && j < end) {
            const uint32_t row = a.list[j];
            const int4 rc = ((const int4*)a.proj.rect)[row];
            auto rel = [](int c, int o) { return min(max(c - o, 0), 8); };
            cov = rel(rc.y, sy * 8) <= w && w < rel(rc.w, sy * 8);
            if (cov) {
                int lo = rel(rc.x, tx0), hi = rel(rc.z, tx0);
                if (a.cull) {
                    const float2 xy = ((const float2*)a.proj.xy)[row];
                    const float4 co = ((const float4*)a.proj.conic_opacity)[row];
                    // the compositing kernels skip power < log(1/(255 alpha_max)); cull with a margin
                    const float R2 = -2.f * __logf(__fdividef(kAlphaMin, co.w)) * 1.0001f + 2e-3f;
                    float4 g0, g1;
                    ellipse_consts(xy.x, xy.y, co.x, co.y, co.z, R2, g0, g1);
                    float ul, ur;
                    if (!ellipse_band_extent(g0, g1, vlo, vhi, ul, ur)) {
                        hi = lo;
                    } else {
                        // tiles [16 tx, 16 tx + 15] meeting [ul, ur]
                        const float fl = ceilf((ul - (float)(kTile - 1)) * (1.f / kTile));
                        const float fh = floorf(ur * (1.f / kTile));
                        lo = max(lo, (int)fminf(fmaxf(fl, -1.f), 1.0e6f) - tx0);
                        hi = min(hi, (int)fminf(fmaxf(fh, -2.f), 1.0e6f) + 1 - tx0);
                    }
                    // the saturation bound needs a*c - b^2 >= 1e-3 a c: the
                    // relative rounding of the power stays far below its size
                    const bool ok = co.x > 0.f && co.z > 0.f && co.x * co.z - co.y * co.y >= 1e-3f * co.x * co.z &&
                                    co.w <= 1.f;
                    const SatRow sr = sat_row(co, xy.x, xy.y, vlo, vhi_img);
                    s_sr0[threadIdx.x] = make_float4(sr.a, sr.B0, sr.B1, sr.C0);
                    s_sr1[threadIdx.x] = make_float4(sr.C1, sr.Bm, sr.Cm, sr.px);
                    s_amax[threadIdx.x] = ok ? co.w : 0.f;
                }
                if (hi > lo) m = (1u << hi) - (1u << lo);
            }
        }
        // the row's queue: stable compaction of the covering entries
        const unsigned bal = __ballot_sync(0xffffffffu, cov);
        if (lane == 0) s_wn[warp] = __popc(bal);
        __syncthreads();
        uint32_t qi = __popc(bal & lt), nq = 0u;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const uint32_t x = s_wn[q];
            qi += q < warp ? x : 0u;
            nq += x;
        }
        if (cov) s_queue[qi] = (unsigned char)threadIdx.x;
        s_m[threadIdx.x] = (unsigned char)m;
        __syncthreads();
        // warp c: tile c of the row, the queue in batches of 32 while its list is open
        uint32_t keep = 0u;  // queue entries listed in tile c
        if (!sat) {
            keep = nq;
            for (uint32_t sb = 0; sb < nq; sb += 32) {
                const uint32_t q = sb + lane;
                bool bit = false;
                uint32_t wt = 0u;
                if (q < nq) {
                    const int e = s_queue[q];
                    bit = (s_m[e] >> warp) & 1u;
                    if (a.cull && bit) {
                        const float am = s_amax[e];
                        if (am > 0.f) {
                            const float4 p0 = s_sr0[e], p1 = s_sr1[e];
                            SatRow sr;
                            sr.a = p0.x; sr.B0 = p0.y; sr.B1 = p0.z; sr.C0 = p0.w;
                            sr.C1 = p1.x; sr.Bm = p1.y; sr.Cm = p1.z; sr.px = p1.w;
                            sr.amax = am;
                            wt = sat_weight(sr, xlo, xhi);
                        }
                    }
                }
                cnt += __popc(__ballot_sync(0xffffffffu, bit));
                if (a.cull) {
                    wsum += __reduce_add_sync(0xffffffffu, wt);
                    if (wsum >= kSatThreshold) {  // the list ends after this batch
                        sat = true;
                        keep = min(sb + 32u, nq);
                        break;
                    }
                }
            }
        }
        if (lane == 0) s_keep[warp] = keep;
        __syncthreads();
        if (j < end) {  // coverage byte of this tile row
            uint32_t byte = 0u;
            if (cov) {
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    if (qi < s_keep[c]) byte |= m & (1u << c);
            }
            reinterpret_cast<unsigned char*>(a.mask + j)[w] = (unsigned char)byte;
        }
        done = __syncthreads_and(sat);
    }
    if (lane == 0) {
        if (ty < TY && tx0 + warp < TX) a.tile_total[a.tile_base[v] + ty * TX + tx0 + warp] = cnt;
        if (sat) atomicOr(&s_sat, 1u << warp);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a.n_head8[8 * gs + w] = row_end - rgs.x;
        reinterpret_cast<unsigned char*>(a.sat_head + gs)[w] = (unsigned char)s_sat;
        // the last CTA to finish plans the tail from every CTA's results
        __threadfence();
        s_last = atomicAdd(a.ticket + 2, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        seg_plan(a, s_wn);
    }
}

// Head pass, writing, of super-tile gs (a CTA of 256 threads, warp w serving
// tile row w): each tile's list starts at the tile's range start and takes, in
// order, the entries of the head whose coverage byte for the tile row lists
// them in the tile.  Runs in the tail pass's writing kernel (k_tile_filter).
__device__ __forceinline__ void head_write(const TileArgs& a, uint32_t gs, uint32_t* s_row, uint2* s_mask,
                                           unsigned char (*s_queue)[256], int lane, int warp, unsigned lt)
{
    int v = 0;
    for (int q = 1; q < a.V; ++q)
        if ((int)gs >= a.super_base[q]) v = q;
    const int ls = (int)gs - a.super_base[v];
    const int sy = ls / a.STX[v], sx = ls - sy * a.STX[v];
    const int TX = a.TX[v], TY = a.TY[v];
    const int ty = sy * 8 + warp;
    const int tx0 = sx * 8;
    const uint2 rgs = a.sranges[gs];
    uint32_t cur[8];  // next slot of each tile's list
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const bool ok = ty < TY && tx0 + k < TX;
        cur[k] = ok ? a.ranges[a.tile_base[v] + ty * TX + tx0 + k].x : 0u;
    }
    const uint32_t end = rgs.x + a.n_head[gs];
    for (uint32_t b = rgs.x; b < end; b += 256) {
        __syncthreads();
        const uint32_t j = b + threadIdx.x;
        if (j < end) {
            s_row[threadIdx.x] = a.list[j];
            s_mask[threadIdx.x] = a.mask[j];
        }
        __syncthreads();
        const int n = (int)min(256u, end - b);
        // the entries listed in some tile of this row, queued in order so
        // that the writes below run on full warps
        int nq = 0;
        if (ty < TY) {
            for (int sb = 0; sb < n; sb += 32) {
                const int e = sb + lane;
                const bool take = e < n && ((warp < 4 ? s_mask[e].x >> (8 * warp) : s_mask[e].y >> (8 * (warp - 4))) &
                                            0xffu) != 0u;
                const unsigned bal = __ballot_sync(0xffffffffu, take);
                if (take) s_queue[warp][nq + __popc(bal & lt)] = (unsigned char)e;
                nq += __popc(bal);
            }
        }
        __syncwarp();
        for (int sb = 0; sb < nq; sb += 32) {
            const int qi = sb + lane;
            const int e = qi < nq ? s_queue[warp][qi] : 0;
            const unsigned m =
                qi < nq ? (warp < 4 ? s_mask[e].x >> (8 * warp) : s_mask[e].y >> (8 * (warp - 4))) & 0xffu : 0u;
            const uint32_t row = s_row[e];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const bool cov = (m >> k) & 1u;
                const unsigned bal = __ballot_sync(0xffffffffu, cov);
                if (cov) {
                    const uint32_t pos = cur[k] + __popc(bal & lt);
                    a.vals_out[pos] = row;
                    if (a.keys_out) a.keys_out[pos] = (uint32_t)(a.tile_base[v] + ty * TX + tx0 + k);
                }
                cur[k] += __popc(bal);
            }
        }
    }
    __syncthreads();
}


// Tail pass: one CTA per segment (kFilterSeg entries) of what the head pass
// left of a super-tile's row list (8x8 tiles): it streams the rows in depth
// order through shared memory; warp w serves tile row w (8 tiles).
// COUNT: warp w keeps a row for the tiles of its rectangle in tile row w that
// its opacity footprint reaches (the footprint enlarged by a margin that covers
// FP32 rounding, so no pixel result changes) and whose list did not end in the
// head, records them as byte w of the entry's coverage word (bit k: tile column
// k of the super-tile) and counts per (segment, tile).  Write pass: each tile's
// list continues contiguously, in order, from the segment's offsets, driven by
// the coverage words alone.
template <bool COUNT>
__global__ void __launch_bounds__(256) k_tile_filter(TileArgs a)
{
    // COUNT: rectangle relative to the super-tile, clamped to [0, 8], one byte
    // per bound (x0, y0, x1, y1); footprint constants
    __shared__ uint32_t s_rect[COUNT ? 256 : 1];
    __shared__ float4 s_g0[COUNT ? 256 : 1], s_g1[COUNT ? 256 : 1];
    __shared__ uint32_t s_row[COUNT ? 1 : 256];
    __shared__ uint2 s_mask[256];
    __shared__ unsigned char s_queue[8][256];  // per tile row: entries of the chunk it has work for
    // COUNT: coverage byte -> four words of two 16-bit column counters (columns 2q, 2q + 1),
    // so that four warp reductions count all eight columns of 32 entries
    __shared__ uint4 s_spread[COUNT ? 256 : 1];
    __shared__ int s_gs;
    __shared__ uint32_t s_g;
    if (status_failed(a.status)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    const uint32_t nseg = a.seg_base[a.total_super];
    // writing pass: the heads' writes (one ticket per super-tile) come first, then the segments
    const uint32_t nhead = COUNT ? 0u : (uint32_t)a.total_super;
    if (COUNT) {
        const unsigned b = threadIdx.x;
        s_spread[b] = make_uint4((b & 1u) | ((b >> 1 & 1u) << 16), (b >> 2 & 1u) | ((b >> 3 & 1u) << 16),
                                 (b >> 4 & 1u) | ((b >> 5 & 1u) << 16), (b >> 6 & 1u) | ((b >> 7 & 1u) << 16));
        __syncthreads();
    }
    for (;;) {
        // segments are taken from a ticket counter: their costs differ, so a
        // fixed assignment leaves SMs idle while others finish
        if (threadIdx.x == 0) {
            const uint32_t tk = atomicAdd(a.ticket + (COUNT ? 1 : 0), 1u);
            s_g = tk;
            const uint32_t sg = tk - nhead;  // wraps below the heads' tickets
            if ((COUNT || tk >= nhead) && sg < nseg) s_gs = (int)a.seg_super[sg];  // super-tile of the segment
        }
        __syncthreads();
        const uint32_t tk = s_g;
        if (tk >= nhead + nseg) break;
        if (!COUNT && tk < nhead) {
            head_write(a, tk, s_row, s_mask, s_queue, lane, warp, lt);
            continue;
        }
        const uint32_t g = tk - nhead;
        const int gs = s_gs;
        int v = 0;
        for (int w = 1; w < a.V; ++w)
            if (gs >= a.super_base[w]) v = w;
        const int ls = gs - a.super_base[v];
        const int sy = ls / a.STX[v], sx = ls - sy * a.STX[v];
        const int TX = a.TX[v], TY = a.TY[v];
        const int ty = sy * 8 + warp;
        const int tx0 = sx * 8;
        const float vlo = (float)(ty * kTile), vhi = vlo + (float)(kTile - 1);
        uint32_t cur[8];
        uint32_t packed[4] = {0u, 0u, 0u, 0u};  // COUNT: column counters, two per word
        // columns whose lists ended in the head (none are added to them here)
        const uint2 sat = a.sat_head[gs];
        const uint32_t done = ((warp < 4 ? sat.x >> (8 * warp) : sat.y >> (8 * (warp - 4))) & 0xffu);
        const uint32_t* off = a.seg_cnt + (size_t)g * 64 + warp * 8;  // (after k_tile_ranges) segment offsets
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const bool ok = ty < TY && tx0 + k < TX;
            cur[k] = (!COUNT && ok) ? a.tile_total[a.tile_base[v] + ty * TX + tx0 + k] + off[k] : 0u;
        }
        const uint2 rgs = a.sranges[gs];
        const uint32_t sb0 = rgs.x + a.n_head[gs] + (g - a.seg_base[gs]) * kFilterSeg;
        const uint2 rg = make_uint2(sb0, min(sb0 + kFilterSeg, rgs.y));
        for (uint32_t b = rg.x; b < rg.y; b += 256) {
            __syncthreads();
            const uint32_t j = b + threadIdx.x;
            if (j < rg.y) {
                const uint32_t row = a.list[j];
                if (COUNT) {
                    const int4 rc = ((const int4*)a.proj.rect)[row];
                    auto rel = [](int c, int o) { return (uint32_t)min(max(c - o, 0), 8); };
                    const uint32_t x0 = rel(rc.x, tx0), y0 = rel(rc.y, sy * 8), x1 = rel(rc.z, tx0),
                                   y1 = rel(rc.w, sy * 8);
                    // does the rectangle reach a tile whose list is still open?
                    const uint32_t cols = (1u << x1) - (1u << x0);
                    bool open = false;
#pragma unroll
                    for (uint32_t r = 0; r < 8; ++r)
                        if (r >= y0 && r < y1)
                            open |= (cols & ~((r < 4 ? sat.x >> (8 * r) : sat.y >> (8 * (r - 4))) & 0xffu)) != 0u;
                    // a row that reaches no open tile is queued by no tile row (y0 = 8, y1 = 0)
                    s_rect[threadIdx.x] = open ? x0 | y0 << 8 | x1 << 16 | y1 << 24 : 8u << 8;
                    s_mask[threadIdx.x] = make_uint2(0u, 0u);
                    if (a.cull && open) {
                        const float2 xy = ((const float2*)a.proj.xy)[row];
                        const float4 co = ((const float4*)a.proj.conic_opacity)[row];
                        // the compositing kernels skip power < log(1/(255 alpha_max)); cull with a margin
                        const float R2 = -2.f * __logf(__fdividef(kAlphaMin, co.w)) * 1.0001f + 2e-3f;
                        float4 g0, g1;
                        ellipse_consts(xy.x, xy.y, co.x, co.y, co.z, R2, g0, g1);
                        s_g0[threadIdx.x] = g0;
                        s_g1[threadIdx.x] = g1;
                    }
                } else {
                    s_row[threadIdx.x] = row;
                    s_mask[threadIdx.x] = a.mask[j];
                }
            }
            __syncthreads();
            if (ty < TY && done != 0xffu) {  // tile rows whose lists all ended in the head have no work
                const int n = (int)min(256u, rg.y - b);
                // the entries this tile row has work for (COUNT: rectangle covers the
                // row; write pass: listed in some tile of the row), queued in order
                // so that the work below runs on full warps
                int nq = 0;
                for (int sb = 0; sb < n; sb += 32) {
                    const int e = sb + lane;
                    bool take = false;
                    if (e < n) {
                        if (COUNT) {
                            const uint32_t rc = s_rect[e];
                            take = (int)(rc >> 8 & 0xffu) <= warp && warp < (int)(rc >> 24);
                        } else {
                            take = ((warp < 4 ? s_mask[e].x >> (8 * warp) : s_mask[e].y >> (8 * (warp - 4))) & 0xffu &
                                    ~done) != 0u;
                        }
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, take);
                    if (take) s_queue[warp][nq + __popc(bal & lt)] = (unsigned char)e;
                    nq += __popc(bal);
                }
                __syncwarp();
                for (int sb = 0; sb < nq; sb += 32) {
                    const int qi = sb + lane;
                    const int e = qi < nq ? s_queue[warp][qi] : 0;
                    unsigned m = 0;  // tile columns of this tile row the entry is listed in
                    if (qi < nq) {
                        if (COUNT) {
                            const uint32_t rc = s_rect[e];
                            int lo = (int)(rc & 0xffu), hi = (int)(rc >> 16 & 0xffu);  // columns of the super-tile
                            if (a.cull) {
                                float ul, ur;
                                if (!ellipse_band_extent(s_g0[e], s_g1[e], vlo, vhi, ul, ur)) {
                                    hi = lo;
                                } else {
                                    // tiles [16 tx, 16 tx + 15] meeting [ul, ur]
                                    const float fl = ceilf((ul - (float)(kTile - 1)) * (1.f / kTile));
                                    const float fh = floorf(ur * (1.f / kTile));
                                    lo = max(lo, (int)fminf(fmaxf(fl, -1.f), 1.0e6f) - tx0);
                                    hi = min(hi, (int)fminf(fmaxf(fh, -2.f), 1.0e6f) + 1 - tx0);
                                }
                            }
                            if (hi > lo) m = ((1u << hi) - (1u << lo)) & ~done;
                            reinterpret_cast<unsigned char*>(&s_mask[e])[warp] = (unsigned char)m;
                        } else {
                            m = (warp < 4 ? s_mask[e].x >> (8 * warp) : s_mask[e].y >> (8 * (warp - 4))) & 0xffu & ~done;
                        }
                    }
                    if (COUNT) {
                        const uint4 w = s_spread[m];
                        packed[0] += __reduce_add_sync(0xffffffffu, w.x);
                        packed[1] += __reduce_add_sync(0xffffffffu, w.y);
                        packed[2] += __reduce_add_sync(0xffffffffu, w.z);
                        packed[3] += __reduce_add_sync(0xffffffffu, w.w);
                    } else {
                        const uint32_t row = s_row[e];
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const bool cov = (m >> k) & 1u;
                            const unsigned bal = __ballot_sync(0xffffffffu, cov);
                            if (cov) {
                                const uint32_t pos = cur[k] + __popc(bal & lt);
                                a.vals_out[pos] = row;
                                if (a.keys_out) a.keys_out[pos] = (uint32_t)(a.tile_base[v] + ty * TX + tx0 + k);
                            }
                            cur[k] += __popc(bal);
                        }
                    }
                }
            }
            if (COUNT) {
                __syncthreads();
                if (j < rg.y) a.mask[j] = s_mask[threadIdx.x];
            }
        }
        if (COUNT) {  // at most kFilterSeg entries per segment: the 16-bit counters do not overflow
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (lane == k) a.seg_cnt[(size_t)g * 64 + warp * 8 + k] = (packed[k >> 1] >> (16 * (k & 1))) & 0xffffu;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------


struct SortLayout {
    int64_t n_rows, capacity;
    int V, tmax, smax;
    bool binned;
    int64_t parts_d, parts_t, parts_scan, n_chunks;
    int64_t total_tiles, total_super;
    int64_t parts_split;
    size_t off_dkeys[2], off_dvals[2], off_offsets, off_chunk, off_scan_lb, off_dlb[2], off_tlb[2], off_tkeys,
        off_tvals, off_hist, off_dhist, off_suptot, off_rlb, off_tickets, off_split_lb, off_total;
    size_t off_vals1, off_sranges, off_ninst1, off_segbase, off_segcnt, off_segsuper, off_nhead, off_sathead,
        off_nhead8, off_mask, off_tord;
    int64_t max_segs;
    size_t bytes;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr int kSuperShift = 3;  // super-tiles of 8 x 8 tiles

SortLayout sort_layout(int64_t n_rows, int64_t capacity, int V, const int* TX, const int* TY, int tile_sort)
{
    SortLayout L{};
    L.n_rows = n_rows;
    L.capacity = capacity;
    L.V = V;
    int tmax = 1, smax = 1;
    for (int v = 0; v < V; ++v) {
        tmax = std::max(tmax, TX[v] * TY[v]);
        const int sx = (TX[v] + 7) >> kSuperShift, sy = (TY[v] + 7) >> kSuperShift;
        smax = std::max(smax, sx * sy);
        L.total_tiles += (int64_t)TX[v] * TY[v];
        L.total_super += (int64_t)sx * sy;
    }
    L.tmax = (tmax + 3) & ~3;
    L.smax = (smax + 3) & ~3;
    // the split packs super-tile coordinates in 10 bits and keeps 9 counters per super-tile and 8 difference
    // grids in shared memory
    int sdiff = 0;
    bool split_ok = true;
    for (int v = 0; v < V; ++v) {
        const int sx = (TX[v] + 7) >> kSuperShift, sy = (TY[v] + 7) >> kSuperShift;
        split_ok = split_ok && sx < 1024 && sy < 1024;
        sdiff = std::max(sdiff, (sx + 1) * (sy + 1));
    }
    split_ok = split_ok && 4 * (9 * (int64_t)L.smax + 8 * (int64_t)sdiff) <= kSplitMaxSmem;
    L.binned = split_ok && (tile_sort == 2 || (tile_sort == 0 && tmax <= kBinMaxTiles));
    L.parts_d = V > 0 ? (int64_t)V * ((n_rows / V + kSortPart - 1) / kSortPart) : 0;  // partitions within views
    L.parts_t = L.binned ? 0 : (capacity + kSortPart - 1) / kSortPart;
    L.parts_scan = (n_rows + kScanPart - 1) / kScanPart;
    L.parts_split = L.binned ? (capacity + kSplitSlots - 1) / kSplitSlots + V : 0;
    L.n_chunks = L.binned ? 1 : (capacity + kDupChunk - 1) / kDupChunk + 1;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align256(o + std::max<size_t>(bytes, 4)); return r; };
    for (int b = 0; b < 2; ++b) L.off_dkeys[b] = take(4 * (size_t)n_rows);
    for (int b = 0; b < 2; ++b) L.off_dvals[b] = take(4 * (size_t)n_rows);
    L.off_offsets = take(4 * (size_t)n_rows);
    L.off_chunk = take(4 * (size_t)L.n_chunks);
    L.off_scan_lb = take(8 * (size_t)std::max<int64_t>(L.parts_scan, 1));
    for (int b = 0; b < 2; ++b) L.off_dlb[b] = take(4 * (size_t)kRadix * std::max<int64_t>(L.parts_d, 1));
    for (int b = 0; b < 2; ++b) L.off_tlb[b] = take(4 * (size_t)kRadix * std::max<int64_t>(L.parts_t, 1));
    L.off_tkeys = take(L.binned ? 4 : 4 * (size_t)capacity);
    L.off_tvals = take(L.binned ? 4 : 4 * (size_t)capacity);
    L.off_hist = take(4 * (size_t)kRadix * 9);
    // zeroed together with hist: the depth digits per view and the super-tile list sizes
    L.off_dhist = take(4 * (size_t)kRadix * 4 * std::max(V, 1));
    L.off_suptot = take(L.binned ? 4 * (size_t)L.total_super : 4);
    L.off_rlb = take(8 * (size_t)((L.total_tiles + kRangeTiles - 1) / kRangeTiles + 1));  // tile ranges' look-back
    L.off_tord = take(2 * kOrderClasses * 4);  // tile-order class counts and cursors
    L.off_tickets = take(4 * 16);
    L.off_split_lb = take(L.binned ? 8 * (size_t)L.smax * std::max<int64_t>(L.parts_split, 1) : 4);
    L.off_total = take(L.binned ? 4 * (size_t)L.total_tiles : 4);
    L.off_vals1 = take(L.binned ? 4 * (size_t)capacity : 4);
    L.off_sranges = take(L.binned ? 8 * (size_t)L.total_super : 4);
    L.off_ninst1 = take(8);
    L.max_segs = L.binned ? (capacity + kFilterSeg - 1) / kFilterSeg + L.total_super : 1;
    L.off_segbase = take(4 * (size_t)(L.total_super + 1));
    L.off_segcnt = take(L.binned ? 4 * 64 * (size_t)L.max_segs : 4);
    L.off_segsuper = take(L.binned ? 4 * (size_t)L.max_segs : 4);
    L.off_nhead = take(4 * (size_t)std::max<int64_t>(L.total_super, 1));
    L.off_sathead = take(8 * (size_t)std::max<int64_t>(L.total_super, 1));
    L.off_nhead8 = take(32 * (size_t)std::max<int64_t>(L.total_super, 1));
    L.off_mask = take(L.binned ? 8 * (size_t)capacity : 4);
    L.bytes = o;
    return L;
}

// resident CTAs per SM of a kernel (grid-stride kernels launch one wave of them)
template <typename Kernel>
static int ctas_per_sm(Kernel kernel, int threads)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, 0) != cudaSuccess || n < 1) n = 1;
    return n;
}

static int sort_ctas_per_sm()
{
    static int cached = 0;
    if (!cached) {
        int n0 = 0, n1 = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n0, k_onesweep<false>, kSortThreads, 0) != cudaSuccess) n0 = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n1, k_onesweep<true>, kSortThreads, 0) != cudaSuccess) n1 = 1;
        cached = std::max(1, std::min(n0, n1));
    }
    return cached;
}


static cudaError_t run_pass(const PassArgs& a, int64_t parts, int resident, cudaStream_t s)
{
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(parts, resident));
    count_launch();
    if (a.ballot_rank)
        k_onesweep<true><<<blocks, kSortThreads, 0, s>>>(a);
    else
        k_onesweep<false><<<blocks, kSortThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bin_sort(const splat_proj& proj, const ViewBatch& vb, const splat_bins& bins, int32_t* status,
                            void* ws, const LaunchCtx& ctx)
{
    const int64_t n_rows = proj.n * vb.V;
    int TXs[SPLAT_MAX_VIEWS], TYs[SPLAT_MAX_VIEWS];
    for (int v = 0; v < vb.V; ++v) {
        TXs[v] = vb.v[v].TX;
        TYs[v] = vb.v[v].TY;
    }
    const SortLayout L = sort_layout(n_rows, bins.capacity, vb.V, TXs, TYs, ctx.tile_sort);
    if (!L.binned && bins.capacity > 0 && !bins.keys) return cudaErrorInvalidValue;
    char* w = (char*)ws;
    auto U = [&](size_t off) { return (uint32_t*)(w + off); };
    cudaStream_t s = ctx.stream;
    cudaError_t err;
    if ((err = cudaMemsetAsync(w + L.off_hist, 0, (L.off_tickets - L.off_hist) + 64, s)) != cudaSuccess) return err;
    if ((err = cudaMemsetAsync(bins.ranges, 0, sizeof(uint32_t) * 2 * (size_t)vb.total_tiles, s)) != cudaSuccess)
        return err;
    if ((err = cudaMemsetAsync(bins.n_instances, 0, sizeof(int64_t), s)) != cudaSuccess) return err;
    if (bins.n_needed && (err = cudaMemsetAsync(bins.n_needed, 0, sizeof(int64_t), s)) != cudaSuccess) return err;
    if (n_rows == 0) return cudaSuccess;
    uint32_t* hist = U(L.off_hist);
    uint32_t* tickets = U(L.off_tickets);
    const int resident = ctx.num_sms * sort_ctas_per_sm();

    // super-tile grids (binned path)
    int super_base[SPLAT_MAX_VIEWS + 1], STX[SPLAT_MAX_VIEWS], STY[SPLAT_MAX_VIEWS];
    int sb = 0;
    for (int v = 0; v < vb.V; ++v) {
        super_base[v] = sb;
        STX[v] = (vb.v[v].TX + 7) >> kSuperShift;
        STY[v] = (vb.v[v].TY + 7) >> kSuperShift;
        sb += STX[v] * STY[v];
    }
    super_base[vb.V] = sb;
    int sdiff = 0;  // words of the largest view's super-tile difference grid
    for (int v = 0; v < vb.V; ++v) sdiff = std::max(sdiff, (STX[v] + 1) * (STY[v] + 1));
    // 1. depth keys + per-view digit counts and (binned) the super-tile list sizes; zero the first depth
    // look-back buffer, the scan's and the split's
    uint32_t* dhist = U(L.off_dhist);
    uint32_t* suptot = U(L.off_suptot);
    {
        DepthArgs a{};
        a.proj = proj;
        a.V = vb.V;
        a.keys = U(L.off_dkeys[0]);
        a.vals = U(L.off_dvals[0]);
        a.dhist = dhist;
        a.super_total = L.binned ? suptot : nullptr;
        for (int v = 0; v < vb.V; ++v) {
            a.super_base[v] = super_base[v];
            a.STX[v] = STX[v];
            a.STY[v] = STY[v];
        }
        a.zero_a = U(L.off_dlb[0]);
        a.n_zero_a = L.parts_d * kRadix;
        a.zero_b = (unsigned long long*)(w + L.off_scan_lb);
        a.n_zero_b = L.parts_scan;
        a.zero_c = (unsigned long long*)(w + L.off_split_lb);
        a.n_zero_c = L.binned ? L.parts_split * L.smax : 0;
        const size_t smem = L.binned ? 4 * (size_t)sdiff : 0;
        static size_t smem_set = 0;
        if (smem > smem_set) {
            if ((err = cudaFuncSetAttribute(k_depth_keys, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
                cudaSuccess)
                return err;
            smem_set = smem;
        }
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_depth_keys, 256, smem) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        a.blocks_per_view = (int)std::max<int64_t>(
            1, std::min<int64_t>((proj.n + 255) / 256, (int64_t)ctx.num_sms * per_sm / vb.V));
        count_launch();
        k_depth_keys<<<vb.V * a.blocks_per_view, 256, smem, s>>>(a);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    // 2. depth passes (buffers 0 -> 1 -> 0 -> 1 -> 0).  Binned: each view's rows sorted in place, giving the
    // (view, depth) order the super-tile split takes.  Radix path: one sort of all rows by depth, so that
    // the rows without tiles come last (the duplication's chunks assume no such row between listed ones)
    const int passes = 4;
    for (int p = 0; p < passes; ++p) {
        PassArgs a{};
        a.keys_in = U(L.off_dkeys[p & 1]);
        a.vals_in = U(L.off_dvals[p & 1]);
        a.keys_out = p + 1 < passes ? U(L.off_dkeys[(p + 1) & 1]) : nullptr;
        a.vals_out = U(L.off_dvals[(p + 1) & 1]);
        a.n_dev = nullptr;
        a.n_host = n_rows;
        a.cap = n_rows;
        a.hist = dhist + (size_t)p * vb.V * kRadix;
        a.lb = U(L.off_dlb[p & 1]);
        a.lb_next = p + 1 < passes ? U(L.off_dlb[(p + 1) & 1]) : nullptr;
        a.ticket = tickets + p;
        a.status = status;
        a.stage = SPLAT_STAGE_DEPTH_SORT;
        a.shift = 8 * p;
        a.spin_limit = ctx.spin_limit;
        a.seg_len = L.binned ? proj.n : 0;
        a.hist_sum = vb.V;
        a.ballot_rank = p < 3;  // the low depth digits take many values in a warp, the top one few
        if ((err = run_pass(a, L.parts_d, resident, s)) != cudaSuccess) return err;
    }
    const uint32_t* rows = U(L.off_dvals[passes & 1]);
    if (L.binned) {
        // 3. super-tile lists.  The scan of the rows' super-tile counts gives each row its first slot and K1;
        // the lists (K1 entries) live in a capacity-sized buffer, so K1 is checked there, before anything is
        // written (K itself is checked by the tile ranges once the tile lists are counted).  Then the stable
        // split of the slots by super-tile.
        {
            ScanArgs a{};
            a.rows = rows;
            a.n_tiles = proj.n_tiles;
            a.rect = (const int4*)proj.rect;
            a.shift = kSuperShift;
            a.n_rows = n_rows;
            a.offsets = U(L.off_offsets);
            a.chunk_row = U(L.off_chunk);
            a.n_chunks_max = 0;
            a.lb = (unsigned long long*)(w + L.off_scan_lb);
            a.ticket = tickets + 4;
            a.n_instances = (int64_t*)(w + L.off_ninst1);
            a.n_needed = nullptr;
            a.capacity = bins.capacity;
            a.status = status;
            a.spin_limit = ctx.spin_limit;
            const int blocks = (int)std::min<int64_t>(L.parts_scan, (int64_t)ctx.num_sms * 4);
            count_launch();
            k_scan_tiles<<<blocks, kScanThreads, 0, s>>>(a);
            if ((err = cudaGetLastError()) != cudaSuccess) return err;
        }
        {
            SplitArgs a{};
            a.proj = proj;
            a.rows = rows;
            a.offsets = U(L.off_offsets);
            a.super_total = suptot;
            a.n_instances = (const int64_t*)(w + L.off_ninst1);
            a.V = vb.V;
            a.n = proj.n;
            a.smax = L.smax;
            a.sdiff = sdiff;
            a.total_super = sb;
            for (int v = 0; v <= vb.V; ++v) a.super_base[v] = super_base[v];
            for (int v = 0; v < vb.V; ++v) {
                a.STX[v] = STX[v];
                a.STY[v] = STY[v];
            }
            a.lb = (unsigned long long*)(w + L.off_split_lb);
            a.max_parts = L.parts_split;
            a.ticket = tickets + 9;
            a.list = U(L.off_vals1);
            a.sranges = (uint2*)(w + L.off_sranges);
            a.status = status;
            a.spin_limit = ctx.spin_limit;
            const size_t smem = 4 * ((size_t)L.smax * 9 + 8 * (size_t)sdiff);
            static size_t smem_set = 0;
            if (smem > smem_set) {
                if ((err = cudaFuncSetAttribute(k_super_split, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)smem)) != cudaSuccess)
                    return err;
                smem_set = smem;
            }
            int per_sm = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_super_split, 256, smem) != cudaSuccess ||
                per_sm < 1)
                per_sm = 1;
            const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(L.parts_split, (int64_t)ctx.num_sms * per_sm));
            count_launch();
            k_super_split<<<blocks, 256, smem, s>>>(a);
            if ((err = cudaGetLastError()) != cudaSuccess) return err;
        }
        // 4. tile level: per-super-tile lists filtered into per-tile lists (see above)
        TileArgs t{};
        t.proj = proj;
        t.V = vb.V;
        t.n_rows = n_rows;
        t.total_tiles = vb.total_tiles;
        for (int v = 0; v < vb.V; ++v) {
            t.tile_base[v] = vb.v[v].tile_base;
            t.TX[v] = vb.v[v].TX;
            t.TY[v] = vb.v[v].TY;
            t.W[v] = vb.v[v].W;
            t.H[v] = vb.v[v].H;
            t.super_base[v] = super_base[v];
            t.STX[v] = STX[v];
        }
        t.tile_base[vb.V] = vb.total_tiles;
        t.super_base[vb.V] = sb;
        t.total_super = sb;
        t.tile_total = U(L.off_total);
        t.list = U(L.off_vals1);
        t.sranges = (const uint2*)(w + L.off_sranges);
        t.ranges = (const uint2*)bins.ranges;
        t.vals_out = bins.vals;
        t.keys_out = bins.keys;
        t.status = status;
        t.stats = ctx.stats;
        t.cull = ctx.tile_cull;
        t.seg_base = U(L.off_segbase);
        t.seg_cnt = U(L.off_segcnt);
        t.seg_super = U(L.off_segsuper);
        t.n_head = U(L.off_nhead);
        t.n_head8 = U(L.off_nhead8);
        t.sat_head = (uint2*)(w + L.off_sathead);
        t.mask = (uint2*)(w + L.off_mask);
        t.ticket = tickets + 10;
        TileRangeArgs tr{};
        tr.lb = (unsigned long long*)(w + L.off_rlb);
        tr.ticket = tickets + 13;
        tr.ranges = (uint2*)bins.ranges;
        tr.K_out = bins.n_instances;
        tr.capacity = bins.capacity;
        tr.K_super = (const int64_t*)(w + L.off_ninst1);
        tr.needed = bins.n_needed;
        tr.cls = bins.tile_order ? U(L.off_tord) : nullptr;
        tr.spin_limit = ctx.spin_limit;
        // the head of each super-tile list in order (each tile's list up to its
        // saturation), the tail in parallel segments, the prefix over head and
        // segments with the ranges, K and the capacity check, then the heads'
        // and segments' writes in one pass
        static const int per_sm_f[2] = {ctas_per_sm(k_tile_filter<false>, 256), ctas_per_sm(k_tile_filter<true>, 256)};
        auto blocks_f = [&](int c) {
            return (int)std::min<int64_t>(L.max_segs + (c ? 0 : sb), (int64_t)ctx.num_sms * per_sm_f[c]);
        };
        count_launch(4);
        k_head_count<<<8 * sb, 256, 0, s>>>(t);
        k_tile_filter<true><<<blocks_f(1), 256, 0, s>>>(t);
        k_tile_ranges<<<(int)((vb.total_tiles + kRangeTiles - 1) / kRangeTiles), 256, 0, s>>>(t, tr);
        k_tile_filter<false><<<blocks_f(0), 256, 0, s>>>(t);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        return launch_tile_order(bins, L.total_tiles, U(L.off_tord), status, ctx, true);
    }
    // 3. radix path: scan of the per-row tile counts in depth order
    {
        ScanArgs a{};
        a.rows = rows;
        a.n_tiles = proj.n_tiles;
        a.rect = (const int4*)proj.rect;
        a.shift = 0;
        a.n_rows = n_rows;
        a.offsets = U(L.off_offsets);
        a.chunk_row = U(L.off_chunk);
        a.n_chunks_max = L.n_chunks;
        a.lb = (unsigned long long*)(w + L.off_scan_lb);
        a.ticket = tickets + 4;
        a.n_instances = bins.n_instances;
        a.n_needed = bins.n_needed;
        a.capacity = bins.capacity;
        a.status = status;
        a.spin_limit = ctx.spin_limit;
        const int blocks = (int)std::min<int64_t>(L.parts_scan, (int64_t)ctx.num_sms * 4);
        count_launch();
        k_scan_tiles<<<blocks, kScanThreads, 0, s>>>(a);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    // 4. radix path: duplicate, tile-digit passes, ranges
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
        a.hist_sum = 1;
        a.lb = U(L.off_tlb[p & 1]);
        a.lb_next = p + 1 < tile_passes ? U(L.off_tlb[(p + 1) & 1]) : nullptr;
        a.ticket = tickets + 5 + p;
        a.status = status;
        a.stage = SPLAT_STAGE_TILE_SORT;
        a.shift = 8 * p;
        a.spin_limit = ctx.spin_limit;
        if ((err = run_pass(a, L.parts_t, resident, s)) != cudaSuccess) return err;
        cur ^= 1;
    }
    {
        const int blocks = ctx.num_sms * 8;
        count_launch();
        k_ranges<<<blocks, 256, 0, s>>>(bins.keys, bins.n_instances, bins.capacity, (uint2*)bins.ranges, status);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    return launch_tile_order(bins, L.total_tiles, U(L.off_tord), status, ctx);
}

size_t bin_sort_workspace(int64_t n_rows, int64_t capacity, int V, const int* TX, const int* TY, int tile_sort)
{
    return sort_layout(n_rows, capacity, V, TX, TY, tile_sort).bytes;
}

}  // namespace splat
