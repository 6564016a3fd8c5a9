// binsort.cu -- sorting stage (Sec. 3.1, Eq. 3): splats, per-tile depth order, tile ranges.
//
// The paper orders splats by a radix sort of (tile, depth) keys.  We run the same LSD
// radix sort but hoist its depth digits in front of the duplication:
//   1. depth keys of the P Gaussians, stable LSD radix sort (4 passes of 8 bits) -> order;
//   2. exclusive scan of the tile counts in that order -> splat offsets, N, capacity check;
//   3. duplication in depth order: splat = (tile id, Gaussian id);
//   4. stable LSD radix sort of the splats by tile id (ceil(log2 tiles / 8) passes);
//   5. tile ranges from adjacent tile-id changes.
// Because every pass is stable and duplication preserves the depth order, the result is the
// (tile, depth, id) order of the 64-bit-key sort, while only 1-2 passes touch the N splats.
// With two tile passes whose high tile bits and Gaussian id fit one 32-bit word together, the first
// pass writes that word alone, the second sorts the words and writes the ids, and the ranges come
// from per-tile counts taken in the second pass's histogram (the low tile byte of a position is its
// digit run in the first pass's output): from the duplication to the ranges 36 instead of 52 bytes
// per splat, and no ranges pass.
//
// Radix sort design (per pass): a fixed grid of G blocks; block b owns one contiguous key
// range.  hist: per-block 256-bin digit counts (+ global digit totals).  scan: one block per
// digit turns the counts into global output offsets.  scatter: each warp ranks its 32-key
// rounds (by __match_any_sync and by ballots, alternately), warps and tiles are chained in order, so
// the pass is stable.
// No block ever waits on another block.
#include <cuda.h>

#include <mutex>
#include <type_traits>

#include "common.cuh"

namespace tcgs {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 8;                       // keys per thread per tile (P-sized passes: 2048 per tile)
constexpr int kItemsSplat = 8;                  // splat passes (16 costs 128 registers and 2 CTAs/SM: slower)
constexpr int kRadix = 256;
constexpr int kMaxBlocks = 1024;
constexpr int kScanBlocks = 1024;

__device__ __forceinline__ uint32_t load_n(uint32_t n_host, const uint32_t* n_dev) {
    return n_dev ? *n_dev : n_host;
}

template <int TI>
__device__ __forceinline__ void block_range(uint32_t n, int G, uint32_t& lo, uint32_t& hi) {
    uint32_t tiles = (n + TI - 1) / TI;
    uint32_t per = (tiles + G - 1) / G;
    uint64_t l = (uint64_t)blockIdx.x * per * TI;
    uint64_t h = l + (uint64_t)per * TI;
    lo = (uint32_t)(l < n ? l : n);
    hi = (uint32_t)(h < n ? h : n);
}

// The lanes of the warp whose kBits-bit value v equals this lane's, among the valid lanes (an invalid
// lane's mask is its own business: the callers give each invalid lane a distinct low value and use
// nothing of it).  One ballot per bit and one for validity.  __match_any_sync alone saturates the
// shared-memory/MIO pipe of the radix scatter, these ballots alone its issue slots; the scatter
// alternates the two by round (bin_sort with match only / ballots only / alternating: 0.2285 / 0.2162
// / 0.2152 ms on the 1080p frame, 12.70 / 11.24 / 10.59 ms on the 605M-splat 4K frame).
template <int kBits>
__device__ __forceinline__ uint32_t warp_peers(uint32_t v, bool valid) {
    uint32_t peers = __ballot_sync(0xffffffffu, valid);
    if (!valid) peers = ~peers;
#pragma unroll
    for (int b = 0; b < kBits; ++b) {
        const bool bit = (v >> b) & 1u;
        const uint32_t bal = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? bal : ~bal;
    }
    return peers;
}

// Exclusive scan over a block of NT threads; returns the thread's exclusive prefix and the total.
template <typename T, int NT>
__device__ __forceinline__ T block_exclusive_scan(T x, T* warp_sums, T& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) warp_sums[warp] = v;
    __syncthreads();
    if (warp == 0) {
        constexpr int NW = NT / 32;
        T w = lane < NW ? warp_sums[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NW) warp_sums[lane] = w;
    }
    __syncthreads();
    T before = warp > 0 ? warp_sums[warp - 1] : T(0);
    total = warp_sums[NT / 32 - 1];
    __syncthreads();
    return before + v - x;
}

// ---------------------------------------------------------------- radix sort passes

// Per-block digit counts of one pass over a contiguous key range (+ global digit totals).
// kTileCount (second pass of the packed tile sort): the keys are packed words (tile >> 8, id), whose
// low tile byte is the position's digit in the first pass's output (runs of lo_total[d] keys, in
// digit order), so the block takes its range one such run at a time, and after each run adds its
// per-digit counts to that run's tiles (tile_counts[2 t + 1]) before summing them into the block's.
template <int KI, bool kTileCount = false>
__global__ void __launch_bounds__(kThreads) k_radix_hist(const uint32_t* __restrict__ keys, uint32_t n_host,
                                                         const uint32_t* n_dev, int shift, uint32_t mask, int G,
                                                         uint32_t* __restrict__ hist,
                                                         uint32_t* __restrict__ digit_total,
                                                         const uint32_t* __restrict__ lo_total,
                                                         uint32_t* __restrict__ tile_counts) {
    pdl_trigger();
    pdl_wait();
    __shared__ uint32_t h[kWarps][kRadix];
    __shared__ uint32_t s_start[kTileCount ? kRadix + 1 : 1];   // first position of each low digit's run
    __shared__ uint32_t s_ws[kWarps];
    const int t = threadIdx.x, warp = t >> 5;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) h[w][t] = 0;
    uint32_t lo, hi;
    block_range<kThreads * KI>(load_n(n_host, n_dev), G, lo, hi);
    uint32_t s = 0;
    if constexpr (kTileCount) {
        uint32_t n_lo;
        s_start[t] = block_exclusive_scan<uint32_t, kThreads>(lo_total[t], s_ws, n_lo);   // ends in a barrier
        if (t == 0) s_start[kRadix] = n_lo;
        __syncthreads();
        for (uint32_t a = lo; a < hi;) {   // uniform over the block
            // the run holding position a: the largest d with s_start[d] <= a (a non-empty run)
            int d = 0, e = kRadix - 1;
            while (d < e) {
                const int m = (d + e + 1) >> 1;
                if (s_start[m] <= a) d = m; else e = m - 1;
            }
            const uint32_t b = s_start[d + 1] < hi ? s_start[d + 1] : hi;
            for (uint32_t i = a + t; i < b; i += kThreads) atomicAdd(&h[warp][(keys[i] >> shift) & mask], 1u);
            __syncthreads();
            uint32_t c = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                c += h[w][t];
                h[w][t] = 0;
            }
            if (c) atomicAdd(&tile_counts[2 * (((uint32_t)t << 8) | (uint32_t)d) + 1], c);   // tile (t, d)
            s += c;
            __syncthreads();
            a = b;
        }
    } else {
        __syncthreads();
        for (uint32_t i = lo + t; i < hi; i += kThreads) atomicAdd(&h[warp][(keys[i] >> shift) & mask], 1u);
        __syncthreads();
#pragma unroll
        for (int w = 0; w < kWarps; ++w) s += h[w][t];
    }
    hist[(size_t)t * G + blockIdx.x] = s;
    if (s) atomicAdd(&digit_total[t], s);
}

// Block d turns row d of hist (the G per-block counts of digit d) into global offsets:
// offset(d, b) = sum_{d' < d} total(d') + sum_{b' < b} count(d, b').
// kTileRanges (second pass of the packed tile sort): digit d is the high byte of the tile id, so
// tiles 256 d .. 256 d + 255 lie in that order from the digit's offset on; block d turns their counts
// (tile_counts[2 t + 1], from the histogram) into [start, end) ranges, [0, 0) for an empty tile.
template <bool kTileRanges = false>
__global__ void __launch_bounds__(kThreads) k_radix_scan(uint32_t* __restrict__ hist,
                                                         const uint32_t* __restrict__ digit_total,
                                                         uint32_t* __restrict__ digit_total_next, int G,
                                                         uint32_t* __restrict__ tile_ranges, int num_tiles) {
    pdl_trigger();
    pdl_wait();
    __shared__ uint32_t ws[kWarps];
    const int d = blockIdx.x, t = threadIdx.x;
    uint32_t tot;
    uint32_t mine = t < d ? digit_total[t] : 0u;
    // base = sum of totals of smaller digits (reuse the scan for a reduction)
    block_exclusive_scan<uint32_t, kThreads>(mine, ws, tot);
    uint32_t run = tot;
    uint32_t* row = hist + (size_t)d * G;
    for (int b0 = 0; b0 < G; b0 += kThreads) {
        int b = b0 + t;
        uint32_t x = b < G ? row[b] : 0u;
        uint32_t chunk;
        uint32_t ex = block_exclusive_scan<uint32_t, kThreads>(x, ws, chunk);
        if (b < G) row[b] = run + ex;
        run += chunk;
    }
    if (d == 0) digit_total_next[t] = 0u;
    if constexpr (kTileRanges) {
        if (d * kRadix < num_tiles) {   // uniform over the block
            const uint32_t tile = (uint32_t)(d * kRadix + t);
            const uint32_t c = tile < (uint32_t)num_tiles ? tile_ranges[2 * tile + 1] : 0u;
            uint32_t sum;
            const uint32_t start = tot + block_exclusive_scan<uint32_t, kThreads>(c, ws, sum);
            if (tile < (uint32_t)num_tiles) {
                tile_ranges[2 * tile] = c ? start : 0u;
                tile_ranges[2 * tile + 1] = c ? start + c : 0u;
            }
        }
    }
}

// Output forms of a scatter pass: key-value pairs; the packed tile sort's first pass (keys are
// tile ids, values Gaussian ids; it writes one word, (tile >> 8) << pack_shift | id, to vals_out); its
// second pass (keys are those words, there are no values; it writes the ids, the low pack_shift bits,
// to vals_out).
enum : int { kScatterPairs = 0, kScatterPackOut = 1, kScatterPackedIn = 2 };

// Stable scatter of one 8-bit digit.  Per tile of kThreads x KI keys: warp-level ranks
// (warp_peers), a per-digit prefix over the warps, keys and values regrouped by digit in
// shared memory, then written out so that consecutive threads write consecutive addresses of each
// digit's run (coalesced).  Keys of the next tile are loaded one tile ahead; a tile's values are
// requested before its keys are ranked.
template <int KI, int kMode = kScatterPairs>
__global__ void __launch_bounds__(kThreads) k_radix_scatter(const uint32_t* __restrict__ keys_in,
                                                            const uint32_t* __restrict__ vals_in,
                                                            uint32_t* __restrict__ keys_out,
                                                            uint32_t* __restrict__ vals_out, uint32_t n_host,
                                                            const uint32_t* n_dev, int shift, uint32_t mask, int G,
                                                            const uint32_t* __restrict__ offsets, int pack_shift) {
    constexpr bool kVals = kMode != kScatterPackedIn;
    pdl_trigger();
    pdl_wait();
    constexpr int TI = kThreads * KI;
    __shared__ uint32_t wcnt[kWarps][kRadix];
    __shared__ uint32_t boff[kRadix];     // next global position of each digit for this block
    __shared__ uint32_t gdelta[kRadix];   // global position of a digit's run minus its tile-local start
    __shared__ uint32_t ws[kWarps];
    __shared__ uint32_t sk[TI], sv[kVals ? TI : 1];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    uint32_t lo, hi;
    block_range<TI>(load_n(n_host, n_dev), G, lo, hi);
    boff[t] = offsets[(size_t)t * G + blockIdx.x];
    const uint32_t lt_mask = (1u << lane) - 1u;
    uint32_t kn[KI];
    auto load_keys = [&](uint32_t tile) {
        const uint32_t base = tile + (uint32_t)warp * (32 * KI);
#pragma unroll
        for (int r = 0; r < KI; ++r) {
            const uint32_t i = base + r * 32 + lane;
            kn[r] = i < hi ? keys_in[i] : 0u;
        }
    };
    if (lo < hi) load_keys(lo);
    for (uint32_t tile = lo; tile < hi; tile += TI) {
        const uint32_t tile_n = hi - tile < (uint32_t)TI ? hi - tile : (uint32_t)TI;
        const uint32_t base = tile + (uint32_t)warp * (32 * KI);
        uint32_t k[KI], pos[KI], v[KI];
#pragma unroll
        for (int r = 0; r < KI; ++r) k[r] = kn[r];
        // this tile's values, requested now so that the loads are in flight during the ranking
#pragma unroll
        for (int r = 0; r < KI; ++r) {
            const uint32_t i = base + r * 32 + lane;
            v[r] = kVals && i < hi ? vals_in[i] : 0u;
        }
        if (tile + TI < hi) load_keys(tile + TI);
#pragma unroll
        for (int w = 0; w < kWarps; ++w) wcnt[w][t] = 0;
        __syncthreads();
        // pos[r] holds (digit << 16) | rank-in-warp, digit 0x100 marking an item past the end
#pragma unroll
        for (int r = 0; r < KI; ++r) {
            const bool valid = base + r * 32 + lane < hi;
            const uint32_t d = valid ? ((k[r] >> shift) & mask) : (0x100u | lane);
            // even rounds on the match unit, odd ones by ballots: the two pipes share the ranking
            const uint32_t peers = (r & 1) == 0 ? __match_any_sync(0xffffffffu, d) : warp_peers<8>(d, valid);
            uint32_t before = 0;
            if (valid) before = wcnt[warp][d];
            __syncwarp();
            if (valid && lane == 31 - __clz(peers)) wcnt[warp][d] = before + __popc(peers);
            __syncwarp();
            pos[r] = ((valid ? d : 0x100u) << 16) | (before + __popc(peers & lt_mask));
        }
        __syncthreads();
        // digit t: the tile's count, the tile-local start of its run, and each warp's start in it
        // (thread t alone touches column t of wcnt until the barrier)
        uint32_t total = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) total += wcnt[w][t];
        uint32_t tile_total;
        const uint32_t ts = block_exclusive_scan<uint32_t, kThreads>(total, ws, tile_total);
        gdelta[t] = boff[t] - ts;   // the write-out reads one word per key (wraps like the sum it stands for)
        uint32_t run = ts;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t c = wcnt[w][t];
            wcnt[w][t] = run;
            run += c;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < KI; ++r) {
            const uint32_t d = pos[r] >> 16;
            if (d < 0x100u) {
                const uint32_t lp = wcnt[warp][d] + (pos[r] & 0xFFFFu);
                sk[lp] = k[r];
                pos[r] = lp;
            } else {
                pos[r] = 0xFFFFFFFFu;
            }
        }
        if constexpr (kVals) {
#pragma unroll
            for (int r = 0; r < KI; ++r) {
                if (pos[r] != 0xFFFFFFFFu) sv[pos[r]] = v[r];
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < KI; ++q) {
            const uint32_t i = (uint32_t)t + (uint32_t)q * kThreads;
            if (i < tile_n) {
                const uint32_t key = sk[i];
                const uint32_t d = (key >> shift) & mask;
                const uint32_t gp = gdelta[d] + i;
                if constexpr (kMode == kScatterPairs) {
                    keys_out[gp] = key;
                    vals_out[gp] = sv[i];
                } else if constexpr (kMode == kScatterPackOut) {
                    vals_out[gp] = ((key >> 8) << pack_shift) | sv[i];
                } else {
                    vals_out[gp] = key & ((1u << pack_shift) - 1u);
                }
            }
        }
        __syncthreads();
        boff[t] += total;
    }
}

// ---------------------------------------------------------------- binning kernels

__device__ __forceinline__ uint32_t orderable_bits(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Exact tile coverage (tcgs_bin_sort_exact): Gaussian g reaches tile t when the least value of its
// conic form over t's 16 x 16 box of pixel centres, in tile-local coordinates, is at most its reach
// limit (the TC renderer's block-mark limit, whose boxes lie inside the tile's).  Per warp, the 32
// Gaussians' parameters are staged in shared memory once; every splat then reads its Gaussian's.
struct Cover {
    float mx, my, a, b, c, ia, ic, lim;
};

__device__ __forceinline__ Cover cover_of(const float* __restrict__ mean2d, const float* __restrict__ conic,
                                          const float* __restrict__ opacity, uint32_t g) {
    Cover v;
    const float2 m = reinterpret_cast<const float2*>(mean2d)[g];
    v.mx = m.x; v.my = m.y;
    v.a = conic[3 * g]; v.b = conic[3 * g + 1]; v.c = conic[3 * g + 2];
    v.lim = reach_limit(__logf(opacity[g]));
    v.ia = __fdividef(1.f, v.a);
    v.ic = __fdividef(1.f, v.c);
    return v;
}

// Gaussian v reaches the tile whose centre is at tile-local offset (lx, ly) from its mean when the
// least value of its conic form over the tile's 16 x 16 pixel-centre box is within its reach limit.
__device__ __forceinline__ bool tile_reached(const Cover& v, float lx, float ly) {
    constexpr float h = 0.5f * (kTile - 1);
    return v.lim >= 0.f && min_q_box_facing(lx, ly, v.a, v.b, v.c, v.ia, v.ic, -h, h, -h, h) <= v.lim;
}

// Row and column of tile kk of a rectangle `w` tiles wide: the quotient from a float product and one
// correction step (exact for kk < 2^22: the product is then within one of kk / w), integer division
// beyond that.
__device__ __forceinline__ void rect_row_col(uint32_t kk, uint32_t w, float inv_w, uint32_t& row, uint32_t& col) {
    if (kk < (1u << 22)) {
        uint32_t q = __float2uint_rz((float)kk * inv_w);
        int32_t r = (int32_t)(kk - q * w);
        if (r < 0) { --q; r += (int32_t)w; }
        if (r >= (int32_t)w) { ++q; r -= (int32_t)w; }
        row = q;
        col = (uint32_t)r;
    } else {
        row = kk / w;
        col = kk - row * w;
    }
}

// Exact coverage, block-cooperative: the kThreads Gaussians of a block (thread t: Gaussian g_t) have
// their rectangles' tiles dealt out over all threads, kThreads splats per round in Gaussian-major,
// row-major order (so a Gaussian with thousands of tiles is spread over the whole block), and the
// passing splats of each round are packed by a block scan.
struct BlockCover {
    Cover cv[kThreads];
    uint4 rect[kThreads];        // x0, y0, width, exclusive prefix of the rectangle sizes
    float inv_w[kThreads];       // 1 / width
    uint32_t wsum[kWarps];
    uint32_t total;
};

// BlockCover with the exact coverage of wide Gaussians by tile rows (see stage_block_exact).
struct BlockCoverRows : BlockCover {
    uint32_t rpre[kThreads];     // exclusive prefix of the row counts
    unsigned long long wsum64[kWarps];
    uint32_t total_rows;
};

// Stages thread t's Gaussian g (valid) and returns its rectangle size; sets bc.total.  COVER: also
// its coverage parameters (exact coverage).
template <bool COVER = true>
__device__ __forceinline__ uint32_t stage_block_cover(BlockCover& bc, const DevCamera& cam, bool valid, uint32_t g,
                                                      const float* __restrict__ mean2d,
                                                      const int32_t* __restrict__ radius,
                                                      const float* __restrict__ conic,
                                                      const float* __restrict__ opacity) {
    const int t = threadIdx.x;
    uint32_t cnt = 0, x0 = 0, y0 = 0, rw = 1;
    Cover cv{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, -1.f};
    if (valid) {
        const float2 m = reinterpret_cast<const float2*>(mean2d)[g];
        const Rect rc = tile_rect(m.x, m.y, radius[g], cam.grid_w, cam.grid_h);
        cnt = rect_count(rc);
        if (cnt) {
            x0 = (uint32_t)rc.x0; y0 = (uint32_t)rc.y0; rw = (uint32_t)(rc.x1 - rc.x0 + 1);
            if (COVER) cv = cover_of(mean2d, conic, opacity, g);
        }
    }
    uint32_t total;
    const uint32_t pre = block_exclusive_scan<uint32_t, kThreads>(cnt, bc.wsum, total);
    if (COVER) bc.cv[t] = cv;
    bc.rect[t] = make_uint4(x0, y0, rw, pre);
    bc.inv_w[t] = 1.f / (float)rw;
    if (t == 0) bc.total = total;
    __syncthreads();
    return cnt;
}

// Calls f(pass, active, owner, tile, leader, cnt, rank) for every splat of the block, kThreads per
// round (every thread, every round; active false past the end).  The lanes of a warp that hold
// splats of the same Gaussian form a run of consecutive lanes: `leader` marks its first lane, `cnt`
// is its number of passing splats and `rank` the number of them on lower lanes.  No barrier: the
// warps of a round do not depend on one another.
template <typename F>
__device__ __forceinline__ void block_cover_splats(BlockCover& bc, uint32_t grid_w, F&& f) {
    const int t = threadIdx.x, lane = t & 31;
    const uint32_t total = bc.total;
    const uint32_t lt = (1u << lane) - 1u, le = (2u << lane) - 1u;   // lanes below / at or below
    for (uint32_t s0 = 0; s0 < total; s0 += kThreads) {
        const uint32_t sidx = s0 + (uint32_t)t;
        const bool active = sidx < total;
        // owner: the last thread whose prefix is <= sidx (binary search over the block's prefixes)
        int owner = 0;
#pragma unroll
        for (int step = kThreads / 2; step > 0; step >>= 1)
            if (bc.rect[owner + step].w <= sidx) owner += step;
        const uint4 r = bc.rect[owner];
        const uint32_t kk = active ? sidx - r.w : 0u;
        uint32_t row, col;
        rect_row_col(kk, r.z, bc.inv_w[owner], row, col);
        const uint32_t ty = r.y + row, tx = r.x + col;
        const Cover& v = bc.cv[owner];
        const float lx = v.mx - (float)(tx * kTile + kTile / 2), ly = v.my - (float)(ty * kTile + kTile / 2);
        const bool pass = active && tile_reached(v, lx, ly);
        const int prev = __shfl_up_sync(0xffffffffu, owner, 1);
        const bool leader = active && (lane == 0 || prev != owner);
        const uint32_t leads = __ballot_sync(0xffffffffu, leader);
        const uint32_t passes = __ballot_sync(0xffffffffu, pass);
        const uint32_t at_or_below = leads & le;
        const int first = at_or_below ? 31 - __clz(at_or_below) : 0;
        const uint32_t above = leads & ~le;
        const uint32_t end_mask = above ? (1u << (__ffs(above) - 1)) - 1u : 0xFFFFFFFFu;
        const uint32_t run = end_mask & ~((1u << first) - 1u);
        f(pass, active, owner, ty * grid_w + tx, leader, (uint32_t)__popc(passes & run),
          (uint32_t)__popc(passes & run & lt), first);
    }
}

// ---- exact coverage by tile rows
//
// In one row of tiles the tiles a Gaussian reaches form an interval: their pixel-centre boxes span
// the same band of rows, and a box meets the convex region {q <= lim} exactly when its x-range meets
// the region's shadow on the x axis within that band.  So each (Gaussian, tile row) is one unit of
// work: the shadow's ends come from the ellipse in closed form, and the per-tile test (tile_reached)
// fixes the interval's end tiles, so the tiles kept are those the per-tile test keeps (whenever they
// form one run, which they do up to FP32 ties at the reach limit).  Narrow rows and degenerate
// conics test every tile of the row and keep the run from the first to the last passing tile.

// Extent of the reach ellipse {q <= lim} about the mean: half-widths W (x) and H (y), the y offset s
// of its leftmost point (the rightmost one is at -s), and det = ac - b^2.  W < 0: scan the row.
struct Reach {
    float W, H, s, det;
};

__device__ __forceinline__ Reach reach_of(const Cover& v) {
    Reach e;
    e.det = __fsub_rn(__fmul_rn(v.a, v.c), __fmul_rn(v.b, v.b));
    e.W = -1.f;
    e.H = e.s = 0.f;
    if (!(e.det > 0.f) || !(v.lim >= 0.f)) return e;
    const float idet = __frcp_rn(e.det);
    const float W = __fsqrt_rn(__fmul_rn(__fmul_rn(v.lim, v.c), idet));
    const float H = __fsqrt_rn(__fmul_rn(__fmul_rn(v.lim, v.a), idet));
    if (!(W < 1e30f) || !(H < 1e30f)) return e;
    e.W = W;
    e.H = H;
    e.s = __fmul_rn(__fmul_rn(v.b, W), v.ic);
    return e;
}

__device__ __forceinline__ int clamp_tile(float f, int lo, int hi) {
    return (int)fminf(fmaxf(f, (float)lo), (float)hi);   // NaN -> lo
}

// Tiles [L, R] (empty when L > R) of rectangle columns [x0, x1] in tile row ty that Gaussian v reaches.
__device__ int2 row_span(const Cover& v, const Reach& e, int ty, int x0, int x1) {
    const int2 none = make_int2(1, 0);
    if (!(v.lim >= 0.f)) return none;
    const float ly = v.my - (float)(ty * kTile + kTile / 2);
    auto test = [&](int tx) { return tile_reached(v, v.mx - (float)(tx * kTile + kTile / 2), ly); };
    auto scan = [&]() {
        int L = x0;
        while (L <= x1 && !test(L)) ++L;
        if (L > x1) return none;
        int R = x1;
        while (R > L && !test(R)) --R;
        return make_int2(L, R);
    };
    if (e.W < 0.f || x1 - x0 < 3) return scan();
    // the shadow [xa, xb] of the ellipse on the x axis within the row's band of pixel centres
    const float yl = __fsub_rn((float)(ty * kTile) + 0.5f, v.my), yh = __fadd_rn(yl, 15.f);
    float Lf = 1.f, Rf = 0.f;   // empty unless the band meets the ellipse
    if (!(yl > e.H || yh < -e.H)) {
        const float alim = __fmul_rn(v.a, v.lim);
        const float dl = fminf(yh, fmaxf(yl, e.s)), dr = fminf(yh, fmaxf(yl, -e.s));
        const float rl = __fsqrt_rn(fmaxf(0.f, __fsub_rn(alim, __fmul_rn(e.det, __fmul_rn(dl, dl)))));
        const float rr = __fsqrt_rn(fmaxf(0.f, __fsub_rn(alim, __fmul_rn(e.det, __fmul_rn(dr, dr)))));
        const float xa = __fmul_rn(__fsub_rn(__fmul_rn(-v.b, dl), rl), v.ia);
        const float xb = __fmul_rn(__fadd_rn(__fmul_rn(-v.b, dr), rr), v.ia);
        // tiles whose box [16 tx + 0.5, 16 tx + 15.5] meets [mx + xa, mx + xb]
        Lf = ceilf(__fmul_rn(__fsub_rn(__fadd_rn(v.mx, xa), 15.5f), 1.f / kTile));
        Rf = floorf(__fmul_rn(__fsub_rn(__fadd_rn(v.mx, xb), 0.5f), 1.f / kTile));
    }
    if (!(Lf <= Rf) || Rf < (float)x0 || Lf > (float)x1) {
        // no shadow in the rectangle: probe the tile holding the point of least q in the band (the
        // least of the minima over x, (det / a) dy^2, is at the dy nearest to 0), grow from there
        const float dyc = fminf(yh, fmaxf(yl, 0.f));
        const float xc = __fadd_rn(v.mx, __fmul_rn(__fmul_rn(-v.b, dyc), v.ia));
        const int c = clamp_tile(floorf(__fmul_rn(xc, 1.f / kTile)), x0, x1);
        if (!test(c)) return none;
        int L = c, R = c;
        while (L > x0 && test(L - 1)) --L;
        while (R < x1 && test(R + 1)) ++R;
        return make_int2(L, R);
    }
    int L = clamp_tile(Lf, x0, x1), R = clamp_tile(Rf, x0, x1);
    if (test(L)) {
        while (L > x0 && test(L - 1)) --L;
    } else {
        int k = L + 1;
        while (k <= R && !test(k)) ++k;
        if (k > R) return scan();
        L = k;
    }
    if (test(R)) {
        while (R < x1 && test(R + 1)) ++R;
    } else {
        int k = R - 1;
        while (k > L && !test(k)) --k;
        R = k;
    }
    return make_int2(L, R);
}

// Gaussians whose rectangle is at least this many tiles wide are covered by rows; the narrower ones
// tile by tile (for them a row costs about as many box tests as it has tiles, plus the row's own
// bookkeeping).
constexpr int kRowMinWidth = 6;
// The row path runs when the caller's splat capacity allows at least this many splats per Gaussian.
constexpr int kRowsCapacityPerGaussian = 32;
// The packed tile sort runs for capacities of at least this many splats: on short lists it gains
// nothing (bin_sort of the 2.3M-splat 1080p frame 0.226 ms either way; 11.6M splats 0.527 -> 0.491 ms;
// 605M splats 15.8 -> 12.7 ms).
constexpr int64_t kPackedTileSortCapacity = (int64_t)1 << 23;
// The binning kernels keep 8 blocks of 256 threads resident per SM (at most 32 registers a thread):
// their tile path is bound by instruction latency and needs all 8; the row path, out of line, is
// held to the same registers.
constexpr int kCoverBlocksPerSm = 8;

// Exact coverage staging: thread t's Gaussian g (valid) is covered by rows when its rectangle is at
// least kRowMinWidth tiles wide, else tile by tile; a Gaussian that reaches no pixel (limit < 0) by
// neither.  bc.rect holds every Gaussian's rectangle (a wide one with a zero tile count), bc.rpre the
// prefix of the wide ones' row counts; one 64-bit scan forms both prefixes (rows in the high word:
// a block's narrow tiles stay below 256 x 5 x 65536 and its rows below 256 x 65536).
__device__ __forceinline__ void stage_block_exact(BlockCoverRows& bc, const DevCamera& cam, bool valid, uint32_t g,
                                                  const float* __restrict__ mean2d,
                                                  const int32_t* __restrict__ radius,
                                                  const float* __restrict__ conic,
                                                  const float* __restrict__ opacity) {
    const int t = threadIdx.x;
    uint32_t tiles = 0, rows = 0, x0 = 0, y0 = 0, rw = 1;
    Cover cv{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, -1.f};
    if (valid) {
        const float2 m = reinterpret_cast<const float2*>(mean2d)[g];
        const Rect rc = tile_rect(m.x, m.y, radius[g], cam.grid_w, cam.grid_h);
        if (rect_count(rc)) {
            cv = cover_of(mean2d, conic, opacity, g);
            if (cv.lim >= 0.f) {
                x0 = (uint32_t)rc.x0; y0 = (uint32_t)rc.y0; rw = (uint32_t)(rc.x1 - rc.x0 + 1);
                if (rw >= (uint32_t)kRowMinWidth) rows = (uint32_t)(rc.y1 - rc.y0 + 1);
                else tiles = rect_count(rc);
            }
        }
    }
    unsigned long long both;
    const unsigned long long pre = block_exclusive_scan<unsigned long long, kThreads>(
        ((unsigned long long)rows << 32) | tiles, bc.wsum64, both);
    bc.cv[t] = cv;
    bc.rect[t] = make_uint4(x0, y0, rw, (uint32_t)pre);
    bc.inv_w[t] = 1.f / (float)rw;
    bc.rpre[t] = (uint32_t)(pre >> 32);
    if (t == 0) {
        bc.total = (uint32_t)both;
        bc.total_rows = (uint32_t)(both >> 32);
    }
    __syncthreads();
}

// Row `rr` (< total_rows) of the block: its Gaussian (thread index).
__device__ __forceinline__ int row_owner(const BlockCoverRows& bc, uint32_t rr) {
    int owner = 0;
#pragma unroll
    for (int step = kThreads / 2; step > 0; step >>= 1)
        if (bc.rpre[owner + step] <= rr) owner += step;
    return owner;
}

// The reached tiles [L, R] of row rr (< total_rows) of the block, and its tile row.
__device__ __forceinline__ int2 block_row_span(const BlockCoverRows& bc, int owner, uint32_t rr, int& ty) {
    const uint4 rc = bc.rect[owner];
    ty = (int)rc.y + (int)(rr - bc.rpre[owner]);
    const Cover& v = bc.cv[owner];
    return row_span(v, reach_of(v), ty, (int)rc.x, (int)(rc.x + rc.z) - 1);
}

// Inclusive sum of v over this lane's run of equal owners (runs are consecutive lanes, owners
// non-decreasing across the warp), and whether the lane ends its run.
__device__ __forceinline__ uint32_t run_inclusive_sum(uint32_t v, int owner, bool active, bool& run_end) {
    const int lane = threadIdx.x & 31;
    const int key = active ? owner : -1 - lane;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, v, d);
        const int o = __shfl_up_sync(0xffffffffu, key, d);
        if (lane >= d && o == key) v += y;
    }
    const int next = __shfl_down_sync(0xffffffffu, key, 1);
    run_end = active && (lane == 31 || next != key);
    return v;
}

// Count pass of the wide Gaussians, row by row: each thread takes one row of a round, and the rows
// of a Gaussian in a warp add their reached tiles with one atomic.  Out of line, so that the tile
// path of the calling kernel keeps its own register allocation.
__device__ __noinline__ void count_rows(const BlockCoverRows& bc, uint32_t* s_cnt) {
    const uint32_t total_rows = bc.total_rows;
    for (uint32_t r0 = 0; r0 < total_rows; r0 += kThreads) {   // no barrier: rounds are independent
        const uint32_t rr = r0 + threadIdx.x;
        const bool active = rr < total_rows;
        int owner = 0;
        uint32_t n = 0;
        if (active) {
            owner = row_owner(bc, rr);
            int ty;
            const int2 sp = block_row_span(bc, owner, rr, ty);
            n = sp.y >= sp.x ? (uint32_t)(sp.y - sp.x + 1) : 0u;
        }
        bool run_end;
        const uint32_t run = run_inclusive_sum(n, owner, active, run_end);
        if (run_end && run) atomicAdd(&s_cnt[owner], run);
    }
}

// Duplication pass of the wide Gaussians, row by row, in rounds of kThreads rows: each warp run of a
// Gaussian's rows claims one slice of the Gaussian's range, then the round's splats are dealt out
// over the threads, kThreads per step, each finding its row by a binary search over the round's
// prefix.  Out of line, so that the tile path of the calling kernel keeps its own register
// allocation.
__device__ __noinline__ void duplicate_rows(const BlockCoverRows& bc, const uint32_t* s_off, uint32_t* s_used,
                                            const uint32_t* s_g, uint32_t grid_w, uint32_t* __restrict__ tile_keys,
                                            uint32_t* __restrict__ vals, uint32_t n_total) {
    __shared__ uint32_t s_rpre[kThreads], s_rpos[kThreads], s_rtile[kThreads], s_rg[kThreads];
    __shared__ uint32_t s_rws[kWarps];
    const uint32_t total_rows = bc.total_rows;
    for (uint32_t r0 = 0; r0 < total_rows; r0 += kThreads) {
        const uint32_t rr = r0 + threadIdx.x;
        const bool active = rr < total_rows;
        int owner = 0;
        uint32_t n = 0, tile0 = 0;
        if (active) {
            owner = row_owner(bc, rr);
            int ty;
            const int2 sp = block_row_span(bc, owner, rr, ty);
            if (sp.y >= sp.x) {
                n = (uint32_t)(sp.y - sp.x + 1);
                tile0 = (uint32_t)ty * grid_w + (uint32_t)sp.x;
            }
        }
        // the run of rows of one Gaussian in this warp claims one slice; each row takes its part
        bool run_end;
        const uint32_t incl = run_inclusive_sum(n, owner, active, run_end);
        uint32_t base = 0;
        if (run_end && incl) base = atomicAdd(&s_used[owner], incl);
        const uint32_t ends = __ballot_sync(0xffffffffu, run_end);
        const int lane = threadIdx.x & 31;
        const uint32_t mine = ends & ~((1u << lane) - 1u);   // this lane's run ends at or above it
        base = __shfl_sync(0xffffffffu, base, mine ? __ffs(mine) - 1 : 31);
        uint32_t round_total;
        const uint32_t pre = block_exclusive_scan<uint32_t, kThreads>(n, s_rws, round_total);
        s_rpre[threadIdx.x] = active ? pre : round_total;
        s_rpos[threadIdx.x] = s_off[owner] + base + (incl - n);
        s_rtile[threadIdx.x] = tile0;
        s_rg[threadIdx.x] = s_g[owner];
        __syncthreads();
        for (uint32_t s0 = 0; s0 < round_total; s0 += kThreads) {
            const uint32_t idx = s0 + threadIdx.x;
            if (idx < round_total) {
                int row = 0;
#pragma unroll
                for (int step = kThreads / 2; step > 0; step >>= 1)
                    if (s_rpre[row + step] <= idx) row += step;
                const uint32_t k = idx - s_rpre[row];
                const uint32_t pos = s_rpos[row] + k;
                if (pos < n_total) {   // always below N: the counts came from the same rows
                    tile_keys[pos] = s_rtile[row] + k;
                    vals[pos] = s_rg[row];
                }
            }
        }
        __syncthreads();
    }
}

// Depth keys, per-Gaussian splat counts, range clearing and the digit totals of pass 0.  The count
// is the rectangle's tile count, or with EXACT the number of its tiles that pass the coverage test
// (added up per Gaussian in shared memory, one atomic per warp run): tile by tile, or with ROWS
// tile by tile for the narrow Gaussians and by rows for the wide ones.
template <bool EXACT, bool ROWS>
__global__ void __launch_bounds__(kThreads, kCoverBlocksPerSm) k_bin_keys(DevCamera cam, int P, const float* __restrict__ mean2d,
                                                       const int32_t* __restrict__ radius,
                                                       const float* __restrict__ depth,
                                                       const float* __restrict__ conic,
                                                       const float* __restrict__ opacity, uint32_t* __restrict__ keys,
                                                       uint32_t* __restrict__ vals, uint32_t* __restrict__ counts,
                                                       uint32_t* __restrict__ ranges, int n_range_words,
                                                       uint32_t* __restrict__ digit_total0) {
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x == 0) digit_total0[threadIdx.x] = 0u;
    if (i < n_range_words) ranges[i] = 0u;
    if (!EXACT) {
        if (i >= P) return;
        const float2 m = reinterpret_cast<const float2*>(mean2d)[i];
        const Rect rc = tile_rect(m.x, m.y, radius[i], cam.grid_w, cam.grid_h);
        const uint32_t c = rect_count(rc);
        counts[i] = c;
        keys[i] = c ? orderable_bits(depth[i]) : 0xFFFFFFFFu;
        vals[i] = (uint32_t)i;
        return;
    }
    __shared__ typename std::conditional<ROWS, BlockCoverRows, BlockCover>::type s_bc;
    __shared__ uint32_t s_cnt[kThreads];
    if ((int)(blockIdx.x * blockDim.x) >= P) return;   // the whole block is past the end
    s_cnt[threadIdx.x] = 0u;
    if constexpr (ROWS) stage_block_exact(s_bc, cam, i < P, (uint32_t)i, mean2d, radius, conic, opacity);
    else stage_block_cover(s_bc, cam, i < P, (uint32_t)i, mean2d, radius, conic, opacity);   // both end with a barrier
    block_cover_splats(s_bc, (uint32_t)cam.grid_w, [&](bool, bool, int owner, uint32_t, bool leader, uint32_t cnt,
                                                      uint32_t, int) {
        if (leader && cnt) atomicAdd(&s_cnt[owner], cnt);
    });
    if constexpr (ROWS) count_rows(s_bc, s_cnt);   // the wide Gaussians, row by row
    __syncthreads();
    if (i < P) {
        const uint32_t c = s_cnt[threadIdx.x];
        counts[i] = c;
        keys[i] = c ? orderable_bits(depth[i]) : 0xFFFFFFFFu;
        vals[i] = (uint32_t)i;
    }
}

// block sums of counts[order[i]] over contiguous ranges
__global__ void __launch_bounds__(kThreads) k_scan_reduce(const uint32_t* __restrict__ counts,
                                                          const uint32_t* __restrict__ order, uint32_t P, int G2,
                                                          unsigned long long* __restrict__ block_sums) {
    pdl_trigger();
    pdl_wait();
    __shared__ unsigned long long ws[kWarps];
    uint32_t per = (P + G2 - 1) / G2;
    uint64_t lo = (uint64_t)blockIdx.x * per, hi = lo + per;
    if (hi > P) hi = P;
    unsigned long long s = 0;
    for (uint64_t i = lo + threadIdx.x; i < hi; i += kThreads) s += counts[order[i]];
    unsigned long long tot;
    block_exclusive_scan<unsigned long long, kThreads>(s, ws, tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_top(unsigned long long* __restrict__ block_sums, int G2,
                                                   int64_t capacity, int64_t* __restrict__ n_splats,
                                                   int32_t* __restrict__ status, uint32_t* __restrict__ n_u32) {
    pdl_trigger();
    pdl_wait();
    __shared__ unsigned long long ws[32];
    int t = threadIdx.x;
    unsigned long long x = t < G2 ? block_sums[t] : 0ull;
    unsigned long long tot;
    unsigned long long ex = block_exclusive_scan<unsigned long long, 1024>(x, ws, tot);
    if (t < G2) block_sums[t] = ex;
    if (t == 0) {
        *n_splats = (int64_t)tot;
        bool ok = tot <= (unsigned long long)capacity;
        *status = ok ? TCGS_OK : TCGS_ERR_CAPACITY;
        *n_u32 = ok ? (uint32_t)tot : 0u;
    }
}

__global__ void __launch_bounds__(kThreads) k_scan_final(const uint32_t* __restrict__ counts,
                                                         const uint32_t* __restrict__ order, uint32_t P, int G2,
                                                         const unsigned long long* __restrict__ block_sums,
                                                         uint32_t* __restrict__ offsets,
                                                         const uint32_t* __restrict__ n_u32) {
    pdl_trigger();
    pdl_wait();
    __shared__ unsigned long long ws[kWarps];
    uint32_t per = (P + G2 - 1) / G2;
    uint64_t lo = (uint64_t)blockIdx.x * per, hi = lo + per;
    if (hi > P) hi = P;
    bool ok = *n_u32 > 0;  // zero splats or capacity exceeded: nothing to place
    unsigned long long run = block_sums[blockIdx.x];
    for (uint64_t c0 = lo; c0 < hi; c0 += kThreads) {
        uint64_t i = c0 + threadIdx.x;
        unsigned long long x = i < hi ? counts[order[i]] : 0ull;
        unsigned long long tot;
        unsigned long long ex = block_exclusive_scan<unsigned long long, kThreads>(x, ws, tot);
        if (ok && i < hi) offsets[i] = (uint32_t)(run + ex);
        run += tot;
    }
}

// Duplication in depth order, one block per 256 consecutive depth-sorted Gaussians: their splats
// occupy one contiguous output range, which the block writes cooperatively, 256 splats per round
// (thread t takes splat t of the round, its Gaussian found by a binary search over the block's
// prefix of rectangle sizes).  Writes are coalesced and a Gaussian with thousands of tiles is spread
// over the whole block.  With EXACT, only the tiles that pass the coverage test are written: those
// of narrow Gaussians tile by tile as above, those of wide ones from their rows' reached intervals
// (the block's range then holds exactly the counted splats).
template <bool EXACT, bool ROWS>
__global__ void __launch_bounds__(kThreads, kCoverBlocksPerSm) k_duplicate(DevCamera cam, uint32_t P, const uint32_t* __restrict__ order,
                                                        const uint32_t* __restrict__ offsets,
                                                        const uint32_t* __restrict__ counts,
                                                        const float* __restrict__ mean2d,
                                                        const int32_t* __restrict__ radius,
                                                        const float* __restrict__ conic,
                                                        const float* __restrict__ opacity,
                                                        uint32_t* __restrict__ tile_keys, uint32_t* __restrict__ vals,
                                                        const uint32_t* __restrict__ n_u32) {
    pdl_wait();
    __shared__ typename std::conditional<ROWS, BlockCoverRows, BlockCover>::type s_bc;
    __shared__ uint32_t s_g[kThreads];
    __shared__ uint32_t s_off[kThreads], s_used[kThreads];
    __shared__ uint32_t s_first;
    const uint32_t n_total = *n_u32;
    if (n_total == 0u || blockIdx.x * blockDim.x >= P) return;   // nothing to place, or past the end
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t g = 0, off = 0;
    bool listed = false;
    if (i < P) {
        g = order[i];
        off = offsets[i];
        listed = counts[g] != 0u;
    }
    // the block's Gaussians are consecutive in depth order, so its splats are contiguous from
    // thread 0's offset
    if (threadIdx.x == 0) s_first = off;
    s_g[threadIdx.x] = g;
    if (EXACT) {
        // A Gaussian's splats fill its own range [offset, offset + count) in any order (the stable
        // tile passes keep only the order between Gaussians): every piece of work claims a slice of
        // it with a shared-memory atomic.
        s_off[threadIdx.x] = off;
        s_used[threadIdx.x] = 0u;
        if constexpr (ROWS) stage_block_exact(s_bc, cam, listed, g, mean2d, radius, conic, opacity);
        else stage_block_cover(s_bc, cam, listed, g, mean2d, radius, conic, opacity);   // both end with a barrier
        // tile by tile: each warp run of a Gaussian claims a slice of its range
        block_cover_splats(s_bc, (uint32_t)cam.grid_w, [&](bool pass, bool, int owner, uint32_t tile, bool leader,
                                                          uint32_t cnt, uint32_t rank, int first) {
            uint32_t base = 0;
            if (leader && cnt) base = atomicAdd(&s_used[owner], cnt);
            base = __shfl_sync(0xffffffffu, base, first);
            const uint32_t pos = s_off[owner] + base + rank;
            if (pass && pos < n_total) {   // always below N: the counts came from the same test
                tile_keys[pos] = tile;
                vals[pos] = s_g[owner];
            }
        });
        if constexpr (ROWS) duplicate_rows(s_bc, s_off, s_used, s_g, (uint32_t)cam.grid_w, tile_keys, vals, n_total);
        return;
    }
    // every rectangle tile is a splat: the block's splats fill [first, first + total) in order
    stage_block_cover<false>(s_bc, cam, listed, g, mean2d, radius, conic, opacity);
    const uint32_t first = s_first, total = s_bc.total;
    for (uint32_t s0 = 0; s0 < total; s0 += kThreads) {
        const uint32_t sidx = s0 + threadIdx.x;
        if (sidx >= total) break;
        int owner = 0;
#pragma unroll
        for (int step = kThreads / 2; step > 0; step >>= 1)
            if (s_bc.rect[owner + step].w <= sidx) owner += step;
        const uint4 r = s_bc.rect[owner];
        const uint32_t kk = sidx - r.w;
        uint32_t row, col;
        rect_row_col(kk, r.z, s_bc.inv_w[owner], row, col);
        const uint32_t ty = r.y + row, tx = r.x + col;
        tile_keys[first + sidx] = ty * (uint32_t)cam.grid_w + tx;
        vals[first + sidx] = s_g[owner];
    }
}

// Tile ranges from tile-id changes of the sorted keys; each thread checks 4 consecutive keys
// (one 16-byte load, the two neighbours from the same cache lines).
__global__ void __launch_bounds__(kThreads) k_ranges(const uint32_t* __restrict__ tile_keys,
                                                     const uint32_t* __restrict__ n_u32,
                                                     uint32_t* __restrict__ ranges) {
    pdl_wait();
    const uint32_t n = *n_u32;
    const uint32_t quads = (n + 3) / 4;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < quads; q += gridDim.x * blockDim.x) {
        const uint32_t i0 = 4 * q;
        uint32_t k[4];
        if (i0 + 3 < n) {
            const uint4 v = reinterpret_cast<const uint4*>(tile_keys)[q];
            k[0] = v.x; k[1] = v.y; k[2] = v.z; k[3] = v.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) k[j] = i0 + j < n ? tile_keys[i0 + j] : 0xFFFFFFFFu;
        }
        const uint32_t prev = i0 > 0 ? tile_keys[i0 - 1] : 0xFFFFFFFFu;
        const uint32_t next = i0 + 4 < n ? tile_keys[i0 + 4] : 0xFFFFFFFFu;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t i = i0 + j;
            if (i < n) {
                const uint32_t before = j == 0 ? prev : k[j - 1];
                const uint32_t after = j == 3 ? next : k[j + 1];
                if (i == 0 || before != k[j]) ranges[2 * k[j]] = i;
                if (i == n - 1 || after != k[j]) ranges[2 * k[j] + 1] = i + 1;
            }
        }
    }
}

// ---------------------------------------------------------------- small views in one CTA

// Views of at most kSmallMaxTiles tiles with at most kSmallMaxP Gaussians and a splat capacity of at
// most kSmallMaxCapacity sort in two single-CTA kernels instead of the multi-block passes, whose
// launches (about 20, each a few microseconds) would otherwise be most of such a frame.  The passes
// are the same stable LSD passes, so the lists are the same.
constexpr int kSmallThreads = 1024;
constexpr int kSmallWarps = kSmallThreads / 32;
constexpr int32_t kSmallMaxP = 8192;
constexpr int64_t kSmallMaxCapacity = 32768;
constexpr int kSmallMaxTiles = kRadix;   // the tile id is then a single 8-bit digit

struct SmallSortSmem {
    uint32_t wcnt[kSmallWarps][kRadix];   // per round: count, then start, of each (warp, digit)
    uint32_t hist[kRadix];                // digit counts of the pass
    uint32_t next[kRadix];                // next output position of each digit
    uint32_t ws[kSmallWarps];
};

// One stable LSD pass of the whole CTA over n items, digit (key >> shift) & mask (mask <= 255):
// digit counts, their exclusive scan, then rounds of 1024 consecutive items, each ranked inside its
// warp by warp_peers and placed after the same digit's items of the lower warps and of the
// earlier rounds.  keys_in and keys_out are distinct buffers; the CTA's last barrier makes the output
// visible to all its threads.
// No __restrict__: the depth kernel reads in one pass what its own threads wrote in the previous one,
// so these loads must not take the read-only path.
__device__ void cta_radix_pass(SmallSortSmem& sm, const uint32_t* kin, const uint32_t* vin, uint32_t* kout,
                               uint32_t* vout, uint32_t n, int shift, uint32_t mask) {
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (t < kRadix) sm.hist[t] = 0u;
    __syncthreads();
    for (uint32_t i = t; i < n; i += kSmallThreads) atomicAdd(&sm.hist[(kin[i] >> shift) & mask], 1u);
    __syncthreads();
    uint32_t total;
    const uint32_t start = block_exclusive_scan<uint32_t, kSmallThreads>(t < kRadix ? sm.hist[t] : 0u, sm.ws, total);
    if (t < kRadix) sm.next[t] = start;
    const uint32_t lt_mask = (1u << lane) - 1u;
    uint32_t* flat = &sm.wcnt[0][0];
    for (uint32_t r0 = 0; r0 < n; r0 += kSmallThreads) {
        for (int j = t; j < kSmallWarps * kRadix; j += kSmallThreads) flat[j] = 0u;
        __syncthreads();
        const uint32_t i = r0 + (uint32_t)t;
        const bool valid = i < n;
        uint32_t k = 0u, v = 0u, d = 0x100u | (uint32_t)lane;   // past the end: a value no digit takes
        if (valid) {
            k = kin[i];
            v = vin[i];
            d = (k >> shift) & mask;
        }
        const uint32_t peers = warp_peers<8>(d, valid);
        const uint32_t rank = __popc(peers & lt_mask);
        if (valid && rank == 0u) sm.wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (t < kRadix) {   // thread t owns digit t: starts over the warps in warp order
            uint32_t run = sm.next[t];
            for (int w = 0; w < kSmallWarps; ++w) {
                const uint32_t c = sm.wcnt[w][t];
                sm.wcnt[w][t] = run;
                run += c;
            }
            sm.next[t] = run;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = sm.wcnt[warp][d] + rank;   // < n: the digit counts sum to n
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
    }
    __syncthreads();
}

// Depth order of the P Gaussians (4 passes, a-buffers -> b -> a -> b -> a), the splat offsets in that
// order, N and the capacity check: the multi-block depth passes and the three scan kernels in one CTA.
__global__ void __launch_bounds__(kSmallThreads) k_small_depth_scan(uint32_t P, uint32_t* dk_a, uint32_t* dv_a,
                                                                    uint32_t* dk_b, uint32_t* dv_b,
                                                                    const uint32_t* __restrict__ counts,
                                                                    uint32_t* __restrict__ offsets, int64_t capacity,
                                                                    int64_t* __restrict__ n_splats,
                                                                    int32_t* __restrict__ status,
                                                                    uint32_t* __restrict__ n_u32) {
    pdl_trigger();
    pdl_wait();
    __shared__ SmallSortSmem sm;
    __shared__ unsigned long long ws64[kSmallWarps];
    for (int pass = 0; pass < 4; ++pass) {
        const bool even = (pass & 1) == 0;
        cta_radix_pass(sm, even ? dk_a : dk_b, even ? dv_a : dv_b, even ? dk_b : dk_a, even ? dv_b : dv_a, P,
                       8 * pass, 0xFFu);
    }
    unsigned long long run = 0;
    for (uint32_t r0 = 0; r0 < P; r0 += kSmallThreads) {
        const uint32_t i = r0 + threadIdx.x;
        unsigned long long tot;
        const unsigned long long ex =
            block_exclusive_scan<unsigned long long, kSmallThreads>(i < P ? counts[dv_a[i]] : 0ull, ws64, tot);
        if (i < P) offsets[i] = (uint32_t)(run + ex);   // read only when N fits the capacity (< 2^32)
        run += tot;
    }
    if (threadIdx.x == 0) {
        *n_splats = (int64_t)run;
        const bool ok = run <= (unsigned long long)capacity;
        *status = ok ? TCGS_OK : TCGS_ERR_CAPACITY;
        *n_u32 = ok ? (uint32_t)run : 0u;
    }
}

// Stable sort of the N splats by tile id (one 8-bit digit) and the tile ranges from its digit counts
// (tiles without splats keep the [0, 0) the key kernel wrote).
__global__ void __launch_bounds__(kSmallThreads) k_small_tile_sort(const uint32_t* kin, const uint32_t* vin,
                                                                   uint32_t* kout, uint32_t* vout,
                                                                   const uint32_t* __restrict__ n_u32, int num_tiles,
                                                                   uint32_t* __restrict__ ranges) {
    pdl_wait();
    __shared__ SmallSortSmem sm;
    cta_radix_pass(sm, kin, vin, kout, vout, *n_u32, 0, 0xFFu);
    const int t = threadIdx.x;
    if (t < num_tiles && sm.hist[t]) {
        ranges[2 * t] = sm.next[t] - sm.hist[t];
        ranges[2 * t + 1] = sm.next[t];
    }
}

// ---------------------------------------------------------------- workspace

struct Workspace {
    uint32_t *dk_a, *dv_a, *dk_b, *dv_b;   // depth sort ping-pong (P)
    uint32_t *counts, *offsets;            // P
    unsigned long long* block_sums;        // kScanBlocks
    uint32_t* hist;                        // 256 * kMaxBlocks
    uint32_t* digit_total;                 // 2 * 256
    uint32_t* n_u32;                       // 1 (+ padding)
    uint32_t *sk_a, *sk_b, *sv_b;          // splat sort buffers (capacity)
    size_t bytes;
};

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

inline Workspace layout(char* base, int64_t P, int64_t cap) {
    Workspace w;
    size_t off = 0;
    auto take = [&](size_t bytes) { char* p = base ? base + off : nullptr; off += align256(bytes); return p; };
    w.dk_a = (uint32_t*)take(4 * P); w.dv_a = (uint32_t*)take(4 * P);
    w.dk_b = (uint32_t*)take(4 * P); w.dv_b = (uint32_t*)take(4 * P);
    w.counts = (uint32_t*)take(4 * P); w.offsets = (uint32_t*)take(4 * P);
    w.block_sums = (unsigned long long*)take(8 * kScanBlocks);
    w.hist = (uint32_t*)take(4 * (size_t)kRadix * kMaxBlocks);
    w.digit_total = (uint32_t*)take(4 * 2 * kRadix);
    w.n_u32 = (uint32_t*)take(256);
    w.sk_a = (uint32_t*)take(4 * cap); w.sk_b = (uint32_t*)take(4 * cap); w.sv_b = (uint32_t*)take(4 * cap);
    w.bytes = off;
    return w;
}

// Blocks of the scatter kernel resident at once on the current device (one full wave: each block
// then walks a contiguous run of tiles, and no second, partly filled wave is left at the end).
// Looked up once per device and instance, under a lock (callers may sort on several devices from
// several host threads).
template <int KI>
inline int resident_sort_blocks() {
    static std::mutex mu;
    static int cached[kMaxDevices] = {};
    DeviceInfo d;
    if (!current_device_info(&d)) return 256;
    std::lock_guard<std::mutex> lock(mu);
    if (cached[d.device] == 0) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_radix_scatter<KI>, kThreads, 0);
        int c = d.sms * (per_sm > 0 ? per_sm : 1);
        if (c < 1) c = 256;
        if (c > kMaxBlocks) c = kMaxBlocks;
        cached[d.device] = c;
    }
    return cached[d.device];
}

template <int KI>
inline int sort_blocks(int64_t n) {
    int64_t tiles = (n + kThreads * KI - 1) / (kThreads * KI);
    if (tiles < 1) tiles = 1;
    const int wave = resident_sort_blocks<KI>();
    return (int)(tiles < wave ? tiles : wave);
}

// One LSD pass on the digit of `bits` (<= 8) bits at `shift`; digit totals ping-pong between two
// 256-word buffers (the scan of a pass zeroes the buffer the next pass accumulates into, after this
// pass's histogram has read it: the previous pass's totals).  kMode and kTiles select the passes of
// the packed tile sort (k_radix_scatter, k_radix_hist, k_radix_scan).
template <int KI, int kMode = kScatterPairs, bool kTiles = false>
inline void radix_pass(const uint32_t* kin, const uint32_t* vin, uint32_t* kout, uint32_t* vout, uint32_t n_host,
                       const uint32_t* n_dev, int shift, int bits, int G, const Workspace& w, int pass,
                       cudaStream_t s, int pack_shift = 0, uint32_t* tile_ranges = nullptr, int num_tiles = 0) {
    uint32_t* tot = w.digit_total + (pass & 1) * kRadix;
    uint32_t* nxt = w.digit_total + ((pass + 1) & 1) * kRadix;
    const uint32_t mask = (1u << bits) - 1u;
    launch_pdl(k_radix_hist<KI, kTiles>, G, kThreads, 0, s, kin, n_host, n_dev, shift, mask, G, w.hist, tot,
               (const uint32_t*)nxt, tile_ranges);
    count_launches(1);
    launch_pdl(k_radix_scan<kTiles>, kRadix, kThreads, 0, s, w.hist, (const uint32_t*)tot, nxt, G, tile_ranges,
               num_tiles);
    count_launches(1);
    launch_pdl(k_radix_scatter<KI, kMode>, G, kThreads, 0, s, kin, vin, kout, vout, n_host, n_dev, shift, mask, G,
               (const uint32_t*)w.hist, pack_shift);
    count_launches(1);
}

}  // namespace
}  // namespace tcgs

extern "C" size_t tcgs_bin_sort_workspace_size(int32_t P, int64_t splat_capacity, int32_t num_tiles) {
    (void)num_tiles;
    if (P < 0 || splat_capacity < 0) return 0;
    return tcgs::layout(nullptr, P, splat_capacity).bytes;
}

namespace tcgs {
namespace {

// The sorting stage; `exact` selects the exact tile coverage (conic and opacity are then read).
tcgs_status bin_sort(const tcgs_camera* cam, int32_t P, const float* mean2d, const int32_t* radius,
                     const float* depth, bool exact, const float* conic, const float* opacity,
                     int64_t splat_capacity, void* workspace, size_t ws_bytes, uint32_t* ids_sorted,
                     uint32_t* tile_ranges, int64_t* n_splats, int32_t* status, cudaStream_t s) {
    if (!valid_camera(cam) || P < 0 || splat_capacity < 0 || splat_capacity > (int64_t)0xFFFFFFFFu)
        return TCGS_ERR_INVALID;
    if (!tile_ranges || !n_splats || !status || (P > 0 && (!mean2d || !radius || !depth)) || !workspace ||
        (splat_capacity > 0 && !ids_sorted))
        return TCGS_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(workspace) & 255) || (reinterpret_cast<uintptr_t>(mean2d) & 7))
        return TCGS_ERR_INVALID;
    DevCamera dc = make_dev_camera(*cam);
    const int num_tiles = dc.grid_w * dc.grid_h;
    Workspace w = layout((char*)workspace, P, splat_capacity);
    if (ws_bytes < w.bytes) return TCGS_ERR_INVALID;

    // keys, counts, range clearing, digit totals of pass 0
    int n_init = P > 2 * num_tiles ? P : 2 * num_tiles;
    if (n_init < kThreads) n_init = kThreads;
    const int kb_blocks = (n_init + kThreads - 1) / kThreads;
    // the row path pays off for wide footprints: chosen when the caller's capacity allows at least
    // kRowsCapacityPerGaussian splats per Gaussian (the lists are the same either way)
    const bool rows = exact && splat_capacity >= (int64_t)kRowsCapacityPerGaussian * P;
    if (rows)
        launch_pdl(k_bin_keys<true, true>, kb_blocks, kThreads, 0, s, dc, P, mean2d, radius, depth, conic, opacity, w.dk_a,
                   w.dv_a, w.counts, tile_ranges, 2 * num_tiles, w.digit_total);
    else if (exact)
        launch_pdl(k_bin_keys<true, false>, kb_blocks, kThreads, 0, s, dc, P, mean2d, radius, depth, conic, opacity, w.dk_a,
                   w.dv_a, w.counts, tile_ranges, 2 * num_tiles, w.digit_total);
    else
        launch_pdl(k_bin_keys<false, false>, kb_blocks, kThreads, 0, s, dc, P, mean2d, radius, depth, conic, opacity, w.dk_a,
                   w.dv_a, w.counts, tile_ranges, 2 * num_tiles, w.digit_total);
    count_launches(1);
    TCGS_CHECK_LAUNCH();
    const bool small = P <= kSmallMaxP && splat_capacity <= kSmallMaxCapacity && num_tiles <= kSmallMaxTiles;
    if (small) {
        // 1-2 in one CTA
        launch_pdl(k_small_depth_scan, 1, kSmallThreads, 0, s, (uint32_t)P, w.dk_a, w.dv_a, w.dk_b, w.dv_b, w.counts,
                   w.offsets, splat_capacity, n_splats, status, w.n_u32);
        count_launches(1);
        TCGS_CHECK_LAUNCH();
        if (splat_capacity == 0 || P == 0) return TCGS_OK;
        // 3. duplication, 4-5. one CTA: the tile sort into ids_sorted and the ranges
        const int dup_blocks = (P + kThreads - 1) / kThreads;
        if (rows)
            launch_pdl(k_duplicate<true, true>, dup_blocks, kThreads, 0, s, dc, (uint32_t)P, w.dv_a, w.offsets,
                       w.counts, mean2d, radius, conic, opacity, w.sk_b, w.sv_b, w.n_u32);
        else if (exact)
            launch_pdl(k_duplicate<true, false>, dup_blocks, kThreads, 0, s, dc, (uint32_t)P, w.dv_a, w.offsets,
                       w.counts, mean2d, radius, conic, opacity, w.sk_b, w.sv_b, w.n_u32);
        else
            launch_pdl(k_duplicate<false, false>, dup_blocks, kThreads, 0, s, dc, (uint32_t)P, w.dv_a, w.offsets,
                       w.counts, mean2d, radius, conic, opacity, w.sk_b, w.sv_b, w.n_u32);
        count_launches(1);
        launch_pdl(k_small_tile_sort, 1, kSmallThreads, 0, s, w.sk_b, w.sv_b, w.sk_a, ids_sorted, w.n_u32, num_tiles,
                   tile_ranges);
        count_launches(1);
        TCGS_CHECK_LAUNCH();
        return TCGS_OK;
    }
    // 1. depth order (4 passes; the result returns to the a-buffers)
    int pass = 0;
    if (P > 0) {
        int Gp = sort_blocks<kItems>(P);
        for (int sh = 0; sh < 32; sh += 8, ++pass) {
            bool even = (pass & 1) == 0;
            radix_pass<kItems>(even ? w.dk_a : w.dk_b, even ? w.dv_a : w.dv_b, even ? w.dk_b : w.dk_a,
                       even ? w.dv_b : w.dv_a, (uint32_t)P, nullptr, sh, 8, Gp, w, pass, s);
        }
        TCGS_CHECK_LAUNCH();
    }
    const uint32_t* order = w.dv_a;
    // 2. offsets, N, capacity check
    int G2 = P < kScanBlocks * 256 ? (P + 255) / 256 : kScanBlocks;
    if (G2 < 1) G2 = 1;
    if (P > 0) {
        launch_pdl(k_scan_reduce, G2, kThreads, 0, s, w.counts, order, (uint32_t)P, G2, w.block_sums);
        count_launches(1);
    } else {
        cudaMemsetAsync(w.block_sums, 0, 8, s);
    }
    launch_pdl(k_scan_top, 1, 1024, 0, s, w.block_sums, G2, splat_capacity, n_splats, status, w.n_u32);
    count_launches(1);
    if (P > 0) {
        launch_pdl(k_scan_final, G2, kThreads, 0, s, w.counts, order, (uint32_t)P, G2, w.block_sums, w.offsets,
                   w.n_u32);
        count_launches(1);
    }
    TCGS_CHECK_LAUNCH();
    if (splat_capacity == 0 || P == 0) return TCGS_OK;
    // 3. duplication into the buffer the first tile pass reads
    int tile_bits = 0;
    while ((1 << tile_bits) < num_tiles) ++tile_bits;
    int tpasses = tile_bits <= 8 ? 1 : (tile_bits <= 16 ? 2 : 3);
    // Two tile passes with the high tile bits and the Gaussian id in one word: the first pass writes
    // (tile >> 8, id) packed, the second sorts those words alone, writes the ids and, from per-tile
    // counts, the ranges (a third of the splat traffic and the ranges pass saved), for capacities of
    // at least kPackedTileSortCapacity splats (the same lists either way).
    int id_bits = 1;
    while (id_bits < 31 && ((int64_t)1 << id_bits) < (int64_t)P) ++id_bits;   // ids 0 .. P - 1
    const bool packed = tpasses == 2 && (tile_bits - 8) + id_bits <= 32 && splat_capacity >= kPackedTileSortCapacity;
    uint32_t* kbuf[2] = {w.sk_a, w.sk_b};
    uint32_t* vbuf[2] = {ids_sorted, w.sv_b};
    int src = packed ? 0 : ((tpasses & 1) ? 1 : 0);
    if (packed) vbuf[0] = w.sv_b;   // the duplication writes (sk_a, sv_b)
    const int dup_blocks = (P + kThreads - 1) / kThreads;
    if (rows)
        launch_pdl(k_duplicate<true, true>, dup_blocks, kThreads, 0, s, dc, (uint32_t)P, order, w.offsets, w.counts,
                   mean2d, radius, conic, opacity, kbuf[src], vbuf[src], w.n_u32);
    else if (exact)
        launch_pdl(k_duplicate<true, false>, dup_blocks, kThreads, 0, s, dc, (uint32_t)P, order, w.offsets, w.counts,
                   mean2d, radius, conic, opacity, kbuf[src], vbuf[src], w.n_u32);
    else
        launch_pdl(k_duplicate<false, false>, dup_blocks, kThreads, 0, s, dc, (uint32_t)P, order, w.offsets, w.counts, mean2d,
                   radius, conic, opacity, kbuf[src], vbuf[src], w.n_u32);
    count_launches(1);
    TCGS_CHECK_LAUNCH();
    // 4. stable sort by tile id, 8 bits per pass (an even split of the tile bits measured slower)
    int Gs = sort_blocks<kItemsSplat>(splat_capacity);
    if (packed) {
        radix_pass<kItemsSplat, kScatterPackOut>(w.sk_a, w.sv_b, nullptr, w.sk_b, 0u, w.n_u32, 0, 8, Gs, w, pass, s,
                                                 id_bits);
        ++pass;
        // 5. ranges from the second pass's per-tile counts (the tile ranges were zeroed by k_bin_keys)
        radix_pass<kItemsSplat, kScatterPackedIn, true>(w.sk_b, nullptr, nullptr, ids_sorted, 0u, w.n_u32, id_bits,
                                                        tile_bits - 8, Gs, w, pass, s, id_bits, tile_ranges,
                                                        num_tiles);
        TCGS_CHECK_LAUNCH();
        return TCGS_OK;
    }
    for (int tp = 0, shift = 0; tp < tpasses; ++tp, ++pass) {
        const int bits = tile_bits - shift < 8 ? tile_bits - shift : 8;
        radix_pass<kItemsSplat>(kbuf[src], vbuf[src], kbuf[src ^ 1], vbuf[src ^ 1], 0u, w.n_u32, shift, bits, Gs, w,
                                pass, s);
        shift += bits;
        src ^= 1;
    }
    TCGS_CHECK_LAUNCH();
    // 5. ranges
    int Gr = sort_blocks<kItemsSplat>(splat_capacity) * 4;
    launch_pdl(k_ranges, Gr, kThreads, 0, s, kbuf[src], w.n_u32, tile_ranges);
    count_launches(1);
    TCGS_CHECK_LAUNCH();
    return TCGS_OK;
}

}  // namespace
}  // namespace tcgs

extern "C" tcgs_status tcgs_bin_sort(const tcgs_camera* cam, int32_t P, const float* mean2d, const int32_t* radius,
                                     const float* depth, int64_t splat_capacity, void* workspace, size_t ws_bytes,
                                     uint32_t* ids_sorted, uint32_t* tile_ranges, int64_t* n_splats,
                                     int32_t* status, tcgs_stream stream) {
    return tcgs::bin_sort(cam, P, mean2d, radius, depth, false, nullptr, nullptr, splat_capacity, workspace, ws_bytes,
                          ids_sorted, tile_ranges, n_splats, status, (cudaStream_t)stream);
}

extern "C" tcgs_status tcgs_bin_sort_exact(const tcgs_camera* cam, int32_t P, const float* mean2d,
                                           const int32_t* radius, const float* depth, const float* conic,
                                           const float* opacity, int64_t splat_capacity, void* workspace,
                                           size_t ws_bytes, uint32_t* ids_sorted, uint32_t* tile_ranges,
                                           int64_t* n_splats, int32_t* status, tcgs_stream stream) {
    if (P > 0 && (!conic || !opacity)) return TCGS_ERR_INVALID;
    return tcgs::bin_sort(cam, P, mean2d, radius, depth, true, conic, opacity, splat_capacity, workspace, ws_bytes,
                          ids_sorted, tile_ranges, n_splats, status, (cudaStream_t)stream);
}

// ---------------------------------------------------------------- longest-first tile order

namespace tcgs {
namespace {

constexpr int kOrderThreads = 1024;
constexpr int kOrderGroups = 33;   // floor(log2(length)) + 1 for lengths 1 .. 2^32 - 1, and 0 for empty

__device__ __forceinline__ int length_group(uint32_t len) { return len ? 32 - __clz(len) : 0; }

// One CTA, a stable counting sort: the groups are laid out from the longest to the empty one, and the
// tiles of a group stay in tile order, so that tiles close on screen, which share Gaussians, stay
// close in the schedule.  Each warp owns a contiguous run of tiles: it counts its run's tiles per
// group, the block turns those counts into the start of every (group, warp) segment, and the warp
// places its tiles in order, ranked among 32 consecutive tiles by warp_peers.  The groups of
// the first kOrderCache tiles are read from global memory once, into shared memory.
constexpr int kOrderCache = 32768;
static_assert(kOrderGroups == 33 && kOrderThreads == 1024, "the scans below take 32 warps and 33 groups");

__global__ void __launch_bounds__(kOrderThreads) k_tile_order(const uint32_t* __restrict__ ranges, uint32_t T,
                                                             uint32_t* __restrict__ order) {
    pdl_wait();
    constexpr int NW = kOrderThreads / 32;
    __shared__ uint8_t s_g[kOrderCache];
    __shared__ uint32_t s_cur[NW][kOrderGroups];   // this warp's tiles of a group, then its next slot there
    __shared__ uint32_t s_base[kOrderGroups];      // a group's total, then its first slot
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const uint32_t cached = T < (uint32_t)kOrderCache ? T : (uint32_t)kOrderCache;
    for (uint32_t i = t; i < cached; i += kOrderThreads)
        s_g[i] = (uint8_t)length_group(ranges[2 * i + 1] - ranges[2 * i]);
    for (int k = t; k < NW * kOrderGroups; k += kOrderThreads) (&s_cur[0][0])[k] = 0u;
    __syncthreads();
    auto group_of = [&](uint64_t i) -> int {
        return i < (uint64_t)kOrderCache ? (int)s_g[i] : length_group(ranges[2 * i + 1] - ranges[2 * i]);
    };
    const uint64_t chunk = ((uint64_t)T + NW - 1) / NW;
    const uint64_t lo = (uint64_t)warp * chunk < T ? (uint64_t)warp * chunk : (uint64_t)T;
    const uint64_t hi = lo + chunk < T ? lo + chunk : (uint64_t)T;
    const uint32_t below = (1u << lane) - 1u;

    for (uint64_t c = lo; c < hi; c += 32) {   // 1: this warp's count per group
        const uint64_t i = c + lane;
        const bool valid = i < hi;
        const int g = valid ? group_of(i) : kOrderGroups + lane;
        const uint32_t peers = warp_peers<6>((uint32_t)g, valid);
        if (valid && lane == __ffs(peers) - 1) s_cur[warp][g] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    for (int g = warp; g < kOrderGroups; g += NW) {   // 2: per group, exclusive prefix over the warps
        const uint32_t v = s_cur[lane][g];
        uint32_t x = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        s_cur[lane][g] = x - v;
        if (lane == 31) s_base[g] = x;
    }
    __syncthreads();
    if (warp == 0) {   // 3: group starts, longest first: lane l takes group 32 - l, group 0 comes last
        const uint32_t v = s_base[32 - lane];
        uint32_t x = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        const uint32_t nonempty = __shfl_sync(0xffffffffu, x, 31);
        __syncwarp();
        s_base[32 - lane] = x - v;
        if (lane == 0) s_base[0] = nonempty;
    }
    __syncthreads();
    for (uint64_t c = lo; c < hi; c += 32) {   // 4: place this warp's tiles in order
        const uint64_t i = c + lane;
        const bool valid = i < hi;
        const int g = valid ? group_of(i) : kOrderGroups + lane;
        const uint32_t peers = warp_peers<6>((uint32_t)g, valid);
        const uint32_t slot = valid ? s_base[g] + s_cur[warp][g] + __popc(peers & below) : 0u;
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) s_cur[warp][g] += __popc(peers);
        __syncwarp();
        if (valid) order[slot] = (uint32_t)i;
    }
}

}  // namespace
}  // namespace tcgs

extern "C" tcgs_status tcgs_tile_order(const tcgs_camera* cam, const uint32_t* tile_ranges, uint32_t* tile_order,
                                       tcgs_stream stream) {
    using namespace tcgs;
    if (!valid_camera(cam) || !tile_ranges || !tile_order) return TCGS_ERR_INVALID;
    const DevCamera dc = make_dev_camera(*cam);
    const uint64_t T = (uint64_t)dc.grid_w * dc.grid_h;
    if (T > 0xFFFFFFFFull) return TCGS_ERR_INVALID;
    launch_pdl(k_tile_order, 1, kOrderThreads, 0, (cudaStream_t)stream, tile_ranges, (uint32_t)T, tile_order);
    count_launches(1);
    TCGS_CHECK_LAUNCH();
    return TCGS_OK;
}

// ---------------------------------------------------------------- work-queue ordering

namespace tcgs {
namespace {

__global__ void __launch_bounds__(kThreads) k_order_keys(const float* __restrict__ cost,
                                                         const uint32_t* __restrict__ items, int n,
                                                         uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                         uint32_t* __restrict__ digit_total0) {
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x == 0) digit_total0[threadIdx.x] = 0u;
    if (i >= n) return;
    keys[i] = ~orderable_bits(cost[i]);   // ascending keys = descending cost
    vals[i] = items[i];
}

struct OrderWs {
    uint32_t *k0, *v0, *k1, *v1, *hist, *digit_total;
    size_t bytes;
};

inline OrderWs order_layout(char* base, int64_t n) {
    OrderWs w;
    size_t off = 0;
    auto take = [&](size_t bytes) { char* p = base ? base + off : nullptr; off += align256(bytes); return p; };
    w.k0 = (uint32_t*)take(4 * n); w.v0 = (uint32_t*)take(4 * n);
    w.k1 = (uint32_t*)take(4 * n); w.v1 = (uint32_t*)take(4 * n);
    w.hist = (uint32_t*)take(4 * (size_t)kRadix * kMaxBlocks);
    w.digit_total = (uint32_t*)take(4 * 2 * kRadix);
    w.bytes = off;
    return w;
}

}  // namespace
}  // namespace tcgs

extern "C" size_t tcgs_sched_order_workspace_size(int32_t n) {
    if (n < 0) return 0;
    return tcgs::order_layout(nullptr, n).bytes;
}

extern "C" tcgs_status tcgs_sched_order(const float* cost, const uint32_t* items, int32_t n, uint32_t* queue_out,
                                        void* workspace, size_t ws_bytes, tcgs_stream stream) {
    using namespace tcgs;
    if (n < 0 || (n > 0 && (!cost || !items || !queue_out || !workspace)) ||
        (reinterpret_cast<uintptr_t>(workspace) & 255))
        return TCGS_ERR_INVALID;
    if (n == 0) return TCGS_OK;
    OrderWs o = order_layout((char*)workspace, n);
    if (ws_bytes < o.bytes) return TCGS_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    launch_pdl(k_order_keys, (n + kThreads - 1) / kThreads, kThreads, 0, s, cost, items, n, o.k0, o.v0, o.digit_total);
    count_launches(1);
    Workspace w = {};
    w.hist = o.hist;
    w.digit_total = o.digit_total;
    const int G = sort_blocks<kItems>(n);
    // 0 -> 1 -> 0 -> 1 -> out
    radix_pass<kItems>(o.k0, o.v0, o.k1, o.v1, (uint32_t)n, nullptr, 0, 8, G, w, 0, s);
    radix_pass<kItems>(o.k1, o.v1, o.k0, o.v0, (uint32_t)n, nullptr, 8, 8, G, w, 1, s);
    radix_pass<kItems>(o.k0, o.v0, o.k1, o.v1, (uint32_t)n, nullptr, 16, 8, G, w, 2, s);
    radix_pass<kItems>(o.k1, o.v1, o.k0, queue_out, (uint32_t)n, nullptr, 24, 8, G, w, 3, s);
    TCGS_CHECK_LAUNCH();
    return TCGS_OK;
}

// ---------------------------------------------------------------- allocation-free variant
//
// The scratch array every tcgs_bin_sort_noalloc call works in.  Host code must not pass its name
// to a kernel (on the host it is only a stand-in symbol): the device address is looked up with
// cudaGetSymbolAddress, with the device current, and passed on as an ordinary workspace pointer.
// The address belongs to the CUDA context the module was loaded in, so it is cached per device
// together with that context and looked up again when the device's current context is another one
// (after cudaDeviceReset, or a release and re-creation of the primary context).
static __device__ __align__(256) unsigned char g_bin_sort_scratch[TCGS_BIN_SORT_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_scratch_mutex;
void* g_scratch_addr[tcgs::kMaxDevices] = {};
CUcontext g_scratch_ctx[tcgs::kMaxDevices] = {};
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
bool g_ctx_fn_looked_up = false;

// The calling thread's current CUDA context (the driver's cuCtxGetCurrent, reached through the
// runtime's entry-point query, so the library needs no link against the driver library), or null.
// Called with g_scratch_mutex held.
CUcontext current_context() {
    if (!g_ctx_fn_looked_up) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(fn);
        g_ctx_fn_looked_up = true;
    }
    CUcontext c = nullptr;
    if (!g_ctx_get_current || g_ctx_get_current(&c) != CUDA_SUCCESS) return nullptr;
    return c;
}
}  // namespace

extern "C" tcgs_status tcgs_bin_sort_noalloc(const tcgs_camera* cam, int32_t P, const float* mean2d,
                                             const int32_t* radius, const float* depth, int64_t splat_capacity,
                                             uint32_t* ids_sorted, uint32_t* tile_ranges, int64_t* n_splats,
                                             int32_t* status, tcgs_stream stream) {
    if (!tcgs::valid_camera(cam) || P < 0 || splat_capacity < 0 || splat_capacity > (int64_t)0xFFFFFFFFu)
        return TCGS_ERR_INVALID;
    const tcgs::DevCamera dc = tcgs::make_dev_camera(*cam);
    const size_t need = tcgs_bin_sort_workspace_size(P, splat_capacity, dc.grid_w * dc.grid_h);
    if (need > (size_t)TCGS_BIN_SORT_NOALLOC_SCRATCH_BYTES) return TCGS_ERR_SCRATCH_LIMIT;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= tcgs::kMaxDevices) return TCGS_ERR_CUDA;
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        CUcontext ctx = current_context();
        if (!g_scratch_addr[dev] || !ctx || ctx != g_scratch_ctx[dev]) {
            void* p = nullptr;   // set-up on this device and context (the lookup also makes the context current)
            if (cudaGetSymbolAddress(&p, g_bin_sort_scratch) != cudaSuccess || !p) return TCGS_ERR_CUDA;
            g_scratch_addr[dev] = p;
            g_scratch_ctx[dev] = current_context();
        }
        scratch = g_scratch_addr[dev];
    }
    return tcgs_bin_sort(cam, P, mean2d, radius, depth, splat_capacity, scratch,
                         (size_t)TCGS_BIN_SORT_NOALLOC_SCRATCH_BYTES, ids_sorted, tile_ranges, n_splats, status,
                         stream);
}
