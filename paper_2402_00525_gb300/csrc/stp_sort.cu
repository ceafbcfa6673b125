// stp_sort.cu -- the sorts of (tile, depth) entries and the per-tile ranges.
//
// Two ways to the same lists: the per-tile sort of appendix B.3 (k_tile_sort, the default;
// described further below) and the global sort of combined keys that StopThePop keeps from
// 3DGS, tile id in the high bits and depth in the low bits (Sec. 2.1, appendix B.3). Both
// give the stable order (ties by Gaussian id) that forward and backward share (Sec. 3.5).
// The global sort (STP_FLAG_GLOBAL_SORT, and stp_sort_pairs) is a stable LSD radix
// sort with 8-bit digits over only the key bits in use (32 depth bits + the bits of the tile
// count), three kernels per digit:
//   hist    -- every block counts the digits of a fixed contiguous range of the input;
//   scan    -- one block turns the [digit][block] counts into exclusive global offsets;
//   scatter -- every block re-reads its range in 4096-item tiles and writes each item to
//              offset[digit][block] + (items of that digit earlier in the block's range).
// Within a tile, warp w owns items [512 w, 512 w + 512) in order and ranks equal digits with
// __match_any_sync, so the write order preserves the input order (stability).
// The grid is fixed (a multiple of the SM count) and the entry count may be read from device
// memory, so the whole sequence needs no host synchronisation and can be graph-captured.
#include <algorithm>

#include <cuda_runtime.h>

#include <mutex>

#include "stp_common.cuh"
#include "stp_kernels.cuh"

namespace stp {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kThreads = 256, kItems = 16, kTileItems = kThreads * kItems;
constexpr int kRadix = 256;
constexpr int kMaxGrid = 1024;

__device__ __forceinline__ long long eff_count(long long nmax, const unsigned long long* n_dev)
{
    if (!n_dev) return nmax;
    const unsigned long long d = *n_dev;
    return d < (unsigned long long)nmax ? (long long)d : nmax;
}

__device__ __forceinline__ void block_range(long long n, int G, int b, long long* beg, long long* end)
{
    const long long tiles = (n + kTileItems - 1) / kTileItems;
    const long long per = (tiles + G - 1) / G;
    *beg = (long long)b * per * kTileItems;
    const long long e = *beg + per * kTileItems;
    *end = e < n ? e : n;
    if (*beg > n) *beg = n;
}

__global__ void __launch_bounds__(kThreads) k_hist(const uint64_t* __restrict__ kin, long long nmax,
                                                   const unsigned long long* n_dev, int shift,
                                                   uint32_t* __restrict__ hist, int G)
{
    __shared__ uint32_t s_h[kThreads / 32][kRadix];
    const int warp = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < (kThreads / 32) * kRadix; k += kThreads) (&s_h[0][0])[k] = 0;
    __syncthreads();
    long long beg, end;
    block_range(eff_count(nmax, n_dev), G, blockIdx.x, &beg, &end);
    for (long long idx = beg + threadIdx.x; idx < end; idx += kThreads) {
        const uint32_t d = (uint32_t)(kin[idx] >> shift) & (kRadix - 1);
        atomicAdd(&s_h[warp][d], 1u);
    }
    __syncthreads();
    uint32_t s = 0;
    for (int w = 0; w < kThreads / 32; w++) s += s_h[w][threadIdx.x];
    hist[threadIdx.x * G + blockIdx.x] = s;
}

__global__ void __launch_bounds__(1024) k_scan(uint32_t* __restrict__ hist, int m)
{
    __shared__ uint32_t ws[32];
    const int per = (m + blockDim.x - 1) / blockDim.x;
    const int b = threadIdx.x * per, e = min(m, b + per);
    uint32_t s = 0;
    for (int k = b; k < e; k++) s += hist[k];
    // block exclusive scan of s
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = s;
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) ws[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint32_t x = ws[lane];
        uint32_t xi = x;
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, xi, d);
            if (lane >= d) xi += y;
        }
        ws[lane] = xi - x;
    }
    __syncthreads();
    uint32_t run = ws[warp] + inc - s;
    for (int k = b; k < e; k++) {
        const uint32_t v = hist[k];
        hist[k] = run;
        run += v;
    }
}

__global__ void __launch_bounds__(kThreads) k_scatter(const uint64_t* __restrict__ kin,
                                                      const uint32_t* __restrict__ vin,
                                                      uint64_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                      long long nmax, const unsigned long long* n_dev,
                                                      int shift, const uint32_t* __restrict__ offs, int G)
{
    __shared__ uint32_t s_run[kRadix];
    __shared__ uint32_t s_base[kRadix];
    __shared__ uint32_t s_wh[kThreads / 32][kRadix];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    long long beg, end;
    block_range(eff_count(nmax, n_dev), G, blockIdx.x, &beg, &end);
    s_run[threadIdx.x] = offs[threadIdx.x * G + blockIdx.x];
    __syncthreads();
    const unsigned lt_mask = lanemask_lt();
    for (long long tb = beg; tb < end; tb += kTileItems) {
        for (int d = lane; d < kRadix; d += 32) s_wh[warp][d] = 0;
        __syncwarp();
        uint64_t k[kItems];
        uint32_t v[kItems], lr[kItems], dg[kItems];
        const long long wb = tb + (long long)warp * (32 * kItems);
#pragma unroll
        for (int j = 0; j < kItems; j++) {
            const long long idx = wb + j * 32 + lane;
            const bool in = idx < end;
            k[j] = in ? kin[idx] : 0ull;
            v[j] = in ? vin[idx] : 0u;
            dg[j] = in ? ((uint32_t)(k[j] >> shift) & (kRadix - 1)) : (uint32_t)kRadix;
        }
#pragma unroll
        for (int j = 0; j < kItems; j++) {
            const uint32_t d = dg[j];
            const unsigned m = __match_any_sync(kFull, d);
            const uint32_t lt = __popc(m & lt_mask);
            const uint32_t cur = d < kRadix ? s_wh[warp][d] : 0u;
            lr[j] = cur + lt;
            __syncwarp();
            if (d < kRadix && lt == 0) s_wh[warp][d] = cur + __popc(m);
            __syncwarp();
        }
        __syncthreads();
        {
            const int d = threadIdx.x;
            uint32_t run = 0;
            for (int w = 0; w < kThreads / 32; w++) {
                const uint32_t c = s_wh[w][d];
                s_wh[w][d] = run;
                run += c;
            }
            s_base[d] = s_run[d];
            s_run[d] += run;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kItems; j++) {
            const uint32_t d = dg[j];
            if (d < kRadix) {
                const uint32_t pos = s_base[d] + s_wh[warp][d] + lr[j];
                kout[pos] = k[j];
                vout[pos] = v[j];
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_ranges(const uint64_t* __restrict__ keys, long long nmax,
                                                const Status* __restrict__ st, int total_tiles,
                                                uint2* __restrict__ ranges)
{
    if (st->error_bits & 1u) return;   // capacity exceeded: the lists are incomplete
    const long long n = eff_count(nmax, &st->num_entries);
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const uint32_t t = (uint32_t)(keys[k] >> 32);
        if (t >= (uint32_t)total_tiles) continue;
        if (k == 0 || (uint32_t)(keys[k - 1] >> 32) != t) ranges[t].x = (uint32_t)k;
        if (k == n - 1 || (uint32_t)(keys[k + 1] >> 32) != t) ranges[t].y = (uint32_t)(k + 1);
    }
}

int sort_grid(long long n)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
    }
    const long long tiles = (n + kTileItems - 1) / kTileItems;
    long long g = 4LL * sms;
    if (g > tiles) g = tiles;
    if (g < 1) g = 1;
    if (g > kMaxGrid) g = kMaxGrid;
    return (int)g;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// ---------------------------------------------------------------- partitioned per-tile sort
// Appendix B.3's alternative to the global sort: Preprocess counted the entries of every tile
// with atomics, a scan gave each tile its range, and Duplicate placed (depth << 32 | id) words
// into the ranges through atomic cursors. One block per tile now sorts its range by (depth,
// id), which reproduces the stable global sort exactly (ties by id), independently of the
// atomic placement order: ranges of at most kSegCap entries by the bucket-and-rank scheme of
// k_tile_sort in shared memory, longer ones (and badly skewed ones) with four stable 8-bit
// passes in place in global memory (the second buffer of the range is the ping-pong partner).
//
// Depth slices (slice_k > 0): a warp stops reading its tile's list once its 32 pixels have
// saturated, which on dense scenes is after a small fraction of the list. So the first pass
// orders only the words of the smallest buckets that together hold at least slice_k of them
// (bucket order is depth order, so they are the list's prefix), publishes that prefix length
// in tile_front and leaves the placed words untouched. The Render queues any warp that would
// need a batch beyond the prefix; the second pass sorts those tiles' whole lists, after which
// the queued warps are rendered again. The result is the whole-list result exactly.
constexpr int kSegThreads = 256, kSegWarps = kSegThreads / 32, kSegCap = 4096;

__device__ __forceinline__ uint32_t seg_digit(unsigned long long x, int shift)
{
    return (uint32_t)(x >> (32 + shift)) & (kRadix - 1);
}

// one stable counting pass of n words from src to dst by the depth digit at `shift`
__device__ void seg_pass(const unsigned long long* src, unsigned long long* dst, int n, int shift,
                         uint32_t (*whist)[kRadix], uint32_t* dtot)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int chunk = (n + kSegWarps - 1) / kSegWarps;
    const int beg = min(n, warp * chunk), end = min(n, beg + chunk);
    const unsigned lt = lanemask_lt();
    for (int d = lane; d < kRadix; d += 32) whist[warp][d] = 0;
    __syncwarp();
    for (int i0 = beg; i0 < end; i0 += 32) {
        const int i = i0 + lane;
        const uint32_t d = i < end ? seg_digit(src[i], shift) : (uint32_t)kRadix;
        const unsigned m = __match_any_sync(kFull, d);
        if (d < kRadix && (m & lt) == 0) whist[warp][d] += __popc(m);
        __syncwarp();
    }
    __syncthreads();
    {   // offsets of (digit, warp): digit-major exclusive scan
        const int d = threadIdx.x;
        uint32_t tot = 0;
        for (int w = 0; w < kSegWarps; w++) tot += whist[w][d];
        dtot[d] = tot;
        __syncthreads();
        if (threadIdx.x < 32) {   // exclusive scan of the 256 digit totals by one warp
            uint32_t v[kRadix / 32], run = 0;
            for (int k = 0; k < kRadix / 32; k++) {
                v[k] = dtot[lane * (kRadix / 32) + k];
                run += v[k];
            }
            uint32_t inc = run;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, inc, o);
                if (lane >= o) inc += y;
            }
            uint32_t base = inc - run;
            for (int k = 0; k < kRadix / 32; k++) {
                dtot[lane * (kRadix / 32) + k] = base;
                base += v[k];
            }
        }
        __syncthreads();
        uint32_t run = dtot[d];
        for (int w = 0; w < kSegWarps; w++) {
            const uint32_t c = whist[w][d];
            whist[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int i0 = beg; i0 < end; i0 += 32) {
        const int i = i0 + lane;
        const unsigned long long x = i < end ? src[i] : 0ull;
        const uint32_t d = i < end ? seg_digit(x, shift) : (uint32_t)kRadix;
        const unsigned m = __match_any_sync(kFull, d);
        const uint32_t rank = __popc(m & lt);
        const uint32_t base = d < kRadix ? whist[warp][d] : 0u;
        if (d < kRadix) dst[base + rank] = x;
        __syncwarp();
        if (d < kRadix && rank == 0) whist[warp][d] = base + __popc(m);
        __syncwarp();
    }
    __syncthreads();
}

// order runs of equal depth by Gaussian id (the low word)
__device__ void seg_fix_ties(unsigned long long* x, int n)
{
    for (int i = threadIdx.x; i < n; i += kSegThreads) {
        const uint32_t hi = (uint32_t)(x[i] >> 32);
        const bool start = (i == 0 || (uint32_t)(x[i - 1] >> 32) != hi) && i + 1 < n && (uint32_t)(x[i + 1] >> 32) == hi;
        if (!start) continue;
        int j = i + 1;
        while (j < n && (uint32_t)(x[j] >> 32) == hi) j++;
        for (int a = i + 1; a < j; a++) {
            const unsigned long long v = x[a];
            int b = a - 1;
            while (b >= i && x[b] > v) {
                x[b + 1] = x[b];
                b--;
            }
            x[b + 1] = v;
        }
    }
    __syncthreads();
}

// Per-tile sort by (depth, id), exact. The (depth, id) words of a tile are distinct, so no
// pass needs to be stable: the tile's depth range is split into NB equal key intervals (one
// shared-memory atomic histogram), the words are scattered into their buckets, and each word's
// place inside its bucket is the number of smaller words there. Buckets hold a few words on
// average. Ranges of at most kSegCap words work in shared memory (1024 buckets); longer ones
// scatter into the range's partner buffer in global memory (4096 buckets). A range whose
// fullest bucket exceeds kBucketMax takes four stable 8-bit radix passes in global memory.
constexpr int kBucketsSmall = 1024, kBucketsLarge = 4096, kBucketMax = 512;

// Bucket of depth word d: the high word of (d - kmin) * mul with mul = min(2^32 - 1,
// floor(NB 2^32 / span)) for a tile's key span, so every bucket is < NB and the map is monotone
// (all a bucket sort needs; the ranks inside buckets make the order exact). One multiply per
// word instead of a 64-bit division.
__device__ __forceinline__ uint32_t bucket_of(uint32_t d, uint32_t kmin, uint32_t mul)
{
    return __umulhi(d - kmin, mul);
}
template <int NB>
__device__ __forceinline__ uint32_t bucket_mul(unsigned long long span)
{
    const unsigned long long m = ((unsigned long long)NB << 32) / span;
    return m > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)m;
}

// The passes over a tile's words are load-latency bound: each thread fetches the four words
// i0 + u*kSegThreads (u < 4) before it uses any of them; words past n read as 0 and are skipped.
constexpr int kSegUnroll = 4;
__device__ __forceinline__ void load_words(const unsigned long long* src, uint32_t i0, uint32_t n,
                                           unsigned long long (&w)[kSegUnroll])
{
#pragma unroll
    for (int u = 0; u < kSegUnroll; u++) {
        const uint32_t i = i0 + u * kSegThreads;
        w[u] = i < n ? src[i] : 0ull;
    }
}

// Histogram + scan of the bucket counts; returns false (nothing written) if a bucket is too
// full. On success bcur[b] holds the start of bucket b.
template <int NB>
__device__ bool bucket_plan(const unsigned long long* src, uint32_t n, uint32_t* bcnt, uint32_t* bcur,
                            uint32_t* red, uint32_t& kmin, uint32_t& mul)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t lo = 0xFFFFFFFFu, hi = 0u;
    for (uint32_t i0 = threadIdx.x; i0 < n; i0 += kSegUnroll * kSegThreads) {
        unsigned long long w[kSegUnroll];
        load_words(src, i0, n, w);
#pragma unroll
        for (int u = 0; u < kSegUnroll; u++) {
            if (i0 + u * kSegThreads >= n) break;
            const uint32_t d = (uint32_t)(w[u] >> 32);
            lo = min(lo, d);
            hi = max(hi, d);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(kFull, lo, o));
        hi = max(hi, __shfl_xor_sync(kFull, hi, o));
    }
    if (lane == 0) {
        red[warp] = lo;
        red[kSegWarps + warp] = hi;
    }
    for (int k = threadIdx.x; k < NB; k += kSegThreads) bcnt[k] = 0;
    __syncthreads();
    lo = red[0];
    hi = red[kSegWarps];
    for (int w = 1; w < kSegWarps; w++) {
        lo = min(lo, red[w]);
        hi = max(hi, red[kSegWarps + w]);
    }
    kmin = lo;
    mul = bucket_mul<NB>((unsigned long long)(hi - lo) + 1ull);
    for (uint32_t i0 = threadIdx.x; i0 < n; i0 += kSegUnroll * kSegThreads) {
        unsigned long long w[kSegUnroll];
        load_words(src, i0, n, w);
#pragma unroll
        for (int u = 0; u < kSegUnroll; u++) {
            if (i0 + u * kSegThreads >= n) break;
            atomicAdd(&bcnt[bucket_of((uint32_t)(w[u] >> 32), kmin, mul)], 1u);
        }
    }
    __syncthreads();
    // exclusive scan of the counts: thread j owns buckets kPer*j .. kPer*j + kPer - 1
    constexpr int kPer = NB / kSegThreads;
    uint32_t c[kPer], sum = 0, mx = 0;
#pragma unroll
    for (int k = 0; k < kPer; k++) {
        c[k] = bcnt[threadIdx.x * kPer + k];
        sum += c[k];
        mx = max(mx, c[k]);
    }
    uint32_t inc = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += y;
    }
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, o));
    __syncthreads();                      // red[] is reused
    if (lane == 31) red[warp] = inc;
    if (lane == 0) red[2 * kSegWarps + warp] = mx;
    __syncthreads();
    uint32_t base = inc - sum, fullest = 0;
    for (int w = 0; w < kSegWarps; w++) {
        if (w < warp) base += red[w];
        fullest = max(fullest, red[2 * kSegWarps + w]);
    }
#pragma unroll
    for (int k = 0; k < kPer; k++) {
        bcur[threadIdx.x * kPer + k] = base;
        base += c[k];
    }
    __syncthreads();
    return fullest <= (uint32_t)kBucketMax;
}

// Scatter the words of buckets 0..cut of src (m of them) into `scat`, then rank each inside its
// bucket: the m smallest words in order (cut = NB - 1, m = n: all of them). With `vals` set,
// the ranked words go straight to the output ids (and, with `keys` set too, to the output
// keys); otherwise to ranked[].
template <int NB>
__device__ void bucket_rank(const unsigned long long* src, unsigned long long* scat, uint32_t n,
                            const uint32_t* bcnt, uint32_t* bcur, uint32_t kmin, uint32_t mul,
                            unsigned long long hi, uint64_t* keys, uint32_t* vals, unsigned long long* ranked,
                            uint32_t cut, uint32_t m)
{
    for (uint32_t i0 = threadIdx.x; i0 < n; i0 += kSegUnroll * kSegThreads) {
        unsigned long long w[kSegUnroll];
        load_words(src, i0, n, w);
#pragma unroll
        for (int u = 0; u < kSegUnroll; u++) {
            if (i0 + u * kSegThreads >= n) break;
            const uint32_t b = bucket_of((uint32_t)(w[u] >> 32), kmin, mul);
            if (b <= cut) scat[atomicAdd(&bcur[b], 1u)] = w[u];
        }
    }
    __syncthreads();
    // bcur[b] is now the end of bucket b (b <= cut)
    for (uint32_t i = threadIdx.x; i < m; i += kSegThreads) {
        const unsigned long long x = scat[i];
        const uint32_t b = bucket_of((uint32_t)(x >> 32), kmin, mul);
        const uint32_t end = bcur[b], beg = end - bcnt[b];
        uint32_t r = beg;
        for (uint32_t j = beg; j < end; j++) r += scat[j] < x;
        if (vals) {
            if (keys) keys[r] = hi | (x >> 32);
            vals[r] = (uint32_t)x;
        } else {
            ranked[r] = x;
        }
    }
}

__device__ __forceinline__ void sort_tile(const PipeArgs& a, const int t, unsigned long long* seg_smem, uint32_t* red)
{
    if (a.status->error_bits & 1u) {
        if (threadIdx.x == 0) a.ranges[t] = make_uint2(0u, 0u);
        return;
    }
    const uint32_t cnt = a.tile_counts[t];
    const uint32_t n = min(a.tile_cursor[t], cnt);
    const uint32_t off = a.tile_offsets[t];
    // Depth slices: the first pass may sort only the prefix of a list longer than slice_k (the
    // placed words stay untouched behind it); the second sorts the whole lists of the tiles whose
    // warps the Render queued.
    bool prefix_ok = false;
    if (a.slice_k) {
        if (a.slice_pass) {
            if (a.tile_redo[t] == 0u) return;
        } else {
            prefix_ok = n > (uint32_t)a.slice_k;
            if (threadIdx.x == 0) a.tile_redo[t] = 0u;
        }
    }
    // the sorted range: m words (m < n: a prefix, which the Render sees through tile_front)
    auto publish = [&](uint32_t m) {
        if (threadIdx.x == 0) {
            a.ranges[t] = make_uint2(off, off + m);
            if (a.slice_k) a.tile_front[t] = m < n ? m : cnt;
        }
    };
    if (n == 0) {
        publish(0);
        return;
    }
    unsigned long long* g0 = (unsigned long long*)a.dup_keys + off;   // placed words (buffer A)
    unsigned long long* g1 = (unsigned long long*)a.keys + off;   // partner (buffer B)
    uint32_t* ov = a.vals + off;
    const unsigned long long hi = (unsigned long long)t << 32;
    // the Render reads only the ids; the (tile, depth) keys are written for inspection only
    uint64_t* okeys = (a.flags & kFlagDebugStats) ? a.keys + off : nullptr;
    uint32_t kmin, mul;
    // smallest prefix of whole buckets holding >= slice_k words: the first bucket whose end
    // (bucket starts bcur after bucket_plan, plus its count) reaches slice_k
    auto prefix_cut = [&](const uint32_t* bcnt, const uint32_t* bcur, int nb, uint32_t& cut, uint32_t& m) {
        cut = (uint32_t)nb - 1u;
        m = n;
        if (!prefix_ok) return;
        uint32_t lo = 0, hb = (uint32_t)nb - 1u;
        while (lo < hb) {
            const uint32_t md = (lo + hb) >> 1;
            if (bcur[md] + bcnt[md] >= (uint32_t)a.slice_k) hb = md; else lo = md + 1;
        }
        cut = lo;
        m = bcur[lo] + bcnt[lo];
    };
    // every thread takes the cut before any thread's scatter moves the bucket cursors
    auto prefix_cut_sync = [&](const uint32_t* bcnt, const uint32_t* bcur, int nb, uint32_t& cut, uint32_t& m) {
        prefix_cut(bcnt, bcur, nb, cut, m);
        __syncthreads();
    };
    if (n <= (uint32_t)kSegCap) {
        uint32_t* bcnt = reinterpret_cast<uint32_t*>(seg_smem + kSegCap);
        uint32_t* bcur = bcnt + kBucketsSmall;
        if (bucket_plan<kBucketsSmall>(g0, n, bcnt, bcur, red, kmin, mul)) {
            uint32_t cut, m;
            prefix_cut_sync(bcnt, bcur, kBucketsSmall, cut, m);
            publish(m);
            bucket_rank<kBucketsSmall>(g0, seg_smem, n, bcnt, bcur, kmin, mul, hi, okeys, ov, nullptr, cut, m);
            return;
        }
    } else {
        uint32_t* bcnt = reinterpret_cast<uint32_t*>(seg_smem);      // 2 x 4096 counters
        uint32_t* bcur = bcnt + kBucketsLarge;
        if (bucket_plan<kBucketsLarge>(g0, n, bcnt, bcur, red, kmin, mul)) {
            if (!okeys) {
                // scatter into the partner range and rank straight into the ids: the placed
                // words stay intact for a later whole sort
                uint32_t cut, m;
                prefix_cut_sync(bcnt, bcur, kBucketsLarge, cut, m);
                publish(m);
                bucket_rank<kBucketsLarge>(g0, g1, n, bcnt, bcur, kmin, mul, hi, nullptr, ov, nullptr, cut, m);
                return;
            }
            // with the inspection keys (written over the partner range): the whole list, ranked
            // back into the placed range and written out
            publish(n);
            bucket_rank<kBucketsLarge>(g0, g1, n, bcnt, bcur, kmin, mul, hi, nullptr, nullptr, g0,
                                       kBucketsLarge - 1, n);
            __syncthreads();
            for (uint32_t i = threadIdx.x; i < n; i += kSegThreads) {
                const unsigned long long v = g0[i];
                okeys[i] = hi | (v >> 32);
                ov[i] = (uint32_t)v;
            }
            return;
        }
    }
    publish(n);
    __syncthreads();                      // shared memory is reused by the radix passes
    // four stable 8-bit passes in global memory, then ties ordered by id
    uint32_t (*whist)[kRadix] = reinterpret_cast<uint32_t (*)[kRadix]>(seg_smem);
    uint32_t* dtot = reinterpret_cast<uint32_t*>(seg_smem) + kSegWarps * kRadix;
    for (int p = 0; p < 4; p++) seg_pass(p % 2 ? g1 : g0, p % 2 ? g0 : g1, (int)n, 8 * p, whist, dtot);
    seg_fix_ties(g0, (int)n);
    for (uint32_t i = threadIdx.x; i < n; i += kSegThreads) {
        const unsigned long long v = g0[i];
        if (okeys) okeys[i] = hi | (v >> 32);
        ov[i] = (uint32_t)v;
    }
}

// One block per tile. The second depth-slice pass (REDO) runs a grid of resident blocks over
// the tiles instead, which returns at once when the Render queued no warp.
template <bool REDO>
__global__ void __launch_bounds__(kSegThreads) k_tile_sort(PipeArgs a)
{
    extern __shared__ unsigned long long seg_smem[];               // [kSegCap] words + counters
    __shared__ uint32_t red[3 * kSegWarps];
    if (!REDO) {
        sort_tile(a, blockIdx.x, seg_smem, red);
        return;
    }
    if (a.status->redo_n == 0u) return;
    for (int t = blockIdx.x; t < a.total_tiles; t += gridDim.x) {
        sort_tile(a, t, seg_smem, red);
        __syncthreads();                  // shared memory is reused by the next tile
    }
}

}  // namespace

size_t sort_hist_bytes() { return align256((size_t)kRadix * kMaxGrid * sizeof(uint32_t)); }

size_t sort_temp_bytes(long long n)
{
    // histogram / offsets of the largest grid, then the ping-pong partner of the output
    return sort_hist_bytes() + align256((size_t)n * sizeof(uint64_t)) + align256((size_t)n * sizeof(uint32_t));
}

static void sort_pass(const uint64_t* sk, const uint32_t* sv, uint64_t* dk, uint32_t* dv, long long n,
                      const unsigned long long* n_dev, int shift, uint32_t* hist, int G, cudaStream_t s)
{
    k_hist<<<G, kThreads, 0, s>>>(sk, n, n_dev, shift, hist, G);
    k_scan<<<1, 1024, 0, s>>>(hist, kRadix * G);
    k_scatter<<<G, kThreads, 0, s>>>(sk, sv, dk, dv, n, n_dev, shift, hist, G);
    note_launches(3);
}

// Sort with explicit scratch: hist holds kRadix x grid counters, (kalt, valt) is the ping-pong
// partner of (kout, vout). Input preserved; the passes alternate between `out` and the partner
// and the last pass writes `out`.
static cudaError_t sort_with(const uint64_t* kin, const uint32_t* vin, uint64_t* kout, uint32_t* vout,
                             long long n, const unsigned long long* n_dev, int key_bits, uint32_t* hist,
                             uint64_t* kalt, uint32_t* valt, cudaStream_t s)
{
    const int passes = (key_bits + 7) / 8;
    if (n == 0 || passes == 0) return cudaSuccess;
    const int G = sort_grid(n);
    const uint64_t* sk = kin;
    const uint32_t* sv = vin;
    for (int p = 0; p < passes; p++) {
        const bool to_out = ((passes - 1 - p) % 2) == 0;
        uint64_t* dk = to_out ? kout : kalt;
        uint32_t* dv = to_out ? vout : valt;
        sort_pass(sk, sv, dk, dv, n, n_dev, 8 * p, hist, G, s);
        sk = dk;
        sv = dv;
    }
    return cudaGetLastError();
}

// Library sort: temp holds the histogram and the ping-pong partner.
cudaError_t sort_pairs(const uint64_t* kin, const uint32_t* vin, uint64_t* kout, uint32_t* vout,
                       long long n, const unsigned long long* n_dev, int key_bits, void* temp,
                       size_t temp_bytes, cudaStream_t s)
{
    if (temp_bytes < sort_temp_bytes(n)) return cudaErrorInvalidValue;
    uint32_t* hist = (uint32_t*)temp;
    uint64_t* kalt = (uint64_t*)((char*)temp + sort_hist_bytes());
    uint32_t* valt = (uint32_t*)((char*)temp + sort_hist_bytes() + align256((size_t)n * sizeof(uint64_t)));
    return sort_with(kin, vin, kout, vout, n, n_dev, key_bits, hist, kalt, valt, s);
}

// ---------------------------------------------------------------- sort without allocation
// Some callers cannot hand the library a device buffer for scratch: code that records work
// into a CUDA graph under stream capture (where a new allocation would not be part of the
// graph), plugins running inside a host framework that owns the device memory pool, and
// real-time loops that must not allocate (an allocation can synchronise the device) after
// start-up. For them the sort's scratch lives in this file-scope device array of fixed size,
// held by every GPU that loads the library until the process exits. All calls share it:
// calls whose work overlaps on the GPU (different streams, or another host thread) race on
// it. Nothing in it needs to start at zero: every call writes the histogram counters and the
// ping-pong keys before it reads them.
constexpr long long kStaticMaxN = 1LL << 20;                          // STP_SORT_STATIC_MAX_N
constexpr long long kStaticGrid = (kStaticMaxN + kTileItems - 1) / kTileItems;
constexpr size_t kStaticHistBytes = ((size_t)kRadix * kStaticGrid * sizeof(uint32_t) + 255) & ~(size_t)255;
constexpr size_t kStaticKeyBytes = (size_t)kStaticMaxN * sizeof(uint64_t);
constexpr size_t kStaticValBytes = (size_t)kStaticMaxN * sizeof(uint32_t);
static __device__ __align__(256) unsigned char g_sort_static_scratch[kStaticHistBytes + kStaticKeyBytes + kStaticValBytes];

constexpr int kMaxDevices = 64;
static void* g_static_addr[kMaxDevices];
static std::mutex g_static_mu;

long long sort_static_max_n() { return kStaticMaxN; }

// Device address of the static scratch on the current device. A call on a stream that is not
// capturing looks the address up again (cudaGetSymbolAddress allocates nothing), so a module
// reloaded after cudaDeviceReset is found at its new place; a call under stream capture uses
// the address of the device's last call outside capture and fails if there was none.
cudaError_t sort_static_scratch(void** out, cudaStream_t s)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(s, &cap)) != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sort_static_scratch);
        if (e != cudaSuccess) return e;
        g_static_addr[dev] = p;
    } else if (!g_static_addr[dev]) {
        return cudaErrorStreamCaptureUnsupported;
    }
    *out = g_static_addr[dev];
    return cudaSuccess;
}

cudaError_t sort_pairs_static(const uint64_t* kin, const uint32_t* vin, uint64_t* kout, uint32_t* vout,
                              long long n, const unsigned long long* n_dev, int key_bits, cudaStream_t s)
{
    if (n < 0 || n > kStaticMaxN || sort_grid(n) > kStaticGrid) return cudaErrorInvalidValue;
    void* base = nullptr;
    cudaError_t e = sort_static_scratch(&base, s);
    if (e != cudaSuccess) return e;
    uint32_t* hist = (uint32_t*)base;
    uint64_t* kalt = (uint64_t*)((char*)base + kStaticHistBytes);
    uint32_t* valt = (uint32_t*)((char*)base + kStaticHistBytes + kStaticKeyBytes);
    return sort_with(kin, vin, kout, vout, n, n_dev, key_bits, hist, kalt, valt, s);
}

// Pipeline sort: Duplicate's output in buffer A = (keys_alt, vals_alt) is sorted by ping-pong
// between A and B = (keys, vals); pass p reads A and writes B for even p. The sorted pairs end
// in B for an odd number of passes and in A otherwise (pipeline_sorted_in_alt()).
bool pipeline_sorted_in_alt(int key_bits) { return ((key_bits + 7) / 8) % 2 == 0; }

cudaError_t pipeline_sort(const PipeArgs& a, cudaStream_t s)
{
    const int passes = (a.key_bits + 7) / 8;
    const long long n = (long long)a.capacity;
    if (n == 0) return cudaSuccess;
    const int G = sort_grid(n);
    uint32_t* hist = (uint32_t*)a.sort_temp;
    const unsigned long long* n_dev = &a.status->num_entries;
    for (int p = 0; p < passes; p++) {
        const bool even = (p % 2) == 0;
        sort_pass(even ? a.keys_alt : a.keys, even ? a.vals_alt : a.vals, even ? a.keys : a.keys_alt,
                  even ? a.vals : a.vals_alt, n, n_dev, 8 * p, hist, G, s);
    }
    return cudaGetLastError();
}

size_t tile_sort_smem_bytes() { return (size_t)kSegCap * sizeof(unsigned long long) + 2 * kBucketsSmall * sizeof(uint32_t); }

cudaError_t launch_tile_sort(const PipeArgs& a, cudaStream_t s)
{
    if (a.total_tiles == 0) return cudaSuccess;
    const size_t smem = tile_sort_smem_bytes();
    cudaError_t e;
    if (a.slice_pass) {      // the second depth-slice pass: resident blocks (40 KB each) over the tiles
        static int set_redo[64];
        if ((e = ensure_smem_limit(k_tile_sort<true>, smem, set_redo, 64)) != cudaSuccess) return e;
        int dev = 0, nsm = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        const unsigned grid = (unsigned)std::min<long long>((long long)nsm * 4, a.total_tiles);
        k_tile_sort<true><<<grid, kSegThreads, smem, s>>>(a);
    } else {
        static int set_dev[64];
        if ((e = ensure_smem_limit(k_tile_sort<false>, smem, set_dev, 64)) != cudaSuccess) return e;
        k_tile_sort<false><<<a.total_tiles, kSegThreads, smem, s>>>(a);
    }
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_ranges(const PipeArgs& a, cudaStream_t s)
{
    cudaMemsetAsync(a.ranges, 0, (size_t)a.total_tiles * sizeof(uint2), s);
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_ranges<<<sms * 8, 256, 0, s>>>(a.skeys, (long long)a.capacity, a.status, a.total_tiles, a.ranges);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace stp
