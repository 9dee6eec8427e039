// gs_sort.cu -- device-wide stable LSD radix sort of (key, u32 value) pairs, 8-bit digits, and
// the per-tile ranges of the sorted pairs.
//
// Sort (the stage FlashGS inherits from 3DGS's CUB SortPairs, Section 2.2).  Three forms share
// one tile body (sort_tile): a CTA loads a tile of 3072 pairs (up to 5120 in the fused form),
// ranks it by digit within each warp (stable: warp-striped load order equals input order; the
// lanes sharing a digit come from a hardware match when the warp's digits form few runs, else
// from shared-memory OR masks), places it in (digit, rank) order in shared memory, learns where
// each digit's run goes, and writes runs of consecutive addresses.
//   * Onesweep (decoupled look-back): the histograms of every digit come from one read of the
//     keys; a tile publishes its per-digit counts in epoch-tagged descriptors (no per-sort
//     clearing) and sums its predecessors' through a two-level look-back -- its own block of 16
//     tiles, then whole-block descriptors that the last tile of each block publishes -- so the
//     last of T tiles that start together waits about 2 + T/256 round trips instead of T/16.
//     Either one kernel per pass with tiles taken in ticket order (k_sort_hist, k_sort_offsets,
//     k_sort_scatter), or the whole sort in one cooperative launch (k_sort_fused): histograms,
//     a grid barrier, then the passes separated by grid barriers, tiles dealt statically.
//   * Reduce-then-scan (k_rts_count, k_rts_scan, k_rts_scatter): per pass, per-tile digit counts,
//     a scan across tiles, then the scatter at the scanned positions; no tile waits on another.
// For 32-bit keys the next tile's keys and values arrive by bulk copy (cp.async.bulk on an
// mbarrier) while the current tile is written out.  Every wait is bounded (waits on other CTAs by
// wait_limit() polls, waits on the CTA's own copies by kSpinLimit) and reports a timeout in the
// frame's status word; a pass or a consumer launched after a timeout writes nothing.
//
// Ranges: the first position of every tile id in the sorted keys, by one pass over the keys or a
// binary search per tile; tile t spans [start[t], start[t+1]).
#include "gs_internal.cuh"

namespace gs {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 12;
static_assert((kSortThreads * kSortItems * 4) % 16 == 0, "bulk copies of a full tile are whole 16-byte units");
constexpr int kSortTile = kSortThreads * kSortItems;
// Items per thread of the per-pass forms' register arrays (they run kSortItems).  The fused sort
// takes as many items (up to kFusedItems, below) as give every CTA one tile of a pass: a second
// tile in some CTAs would double the pass (tiles are at least kSortTile, so the descriptor area
// never grows).
template <class K>
constexpr int kMaxItems = sizeof(K) == 8 ? 14 : kSortItems;
static_assert(32 * 20 < 65536, "in-warp ranks fit 16 bits");
constexpr unsigned kDescAgg = 1u << 30;
constexpr unsigned kDescPrefix = 2u << 30;
constexpr unsigned kDescCount = (1u << 30) - 1;
constexpr int kLookWindow = 16;        // descriptors per look-back round trip
constexpr int kLookBlock = 16;         // tiles per block descriptor
constexpr unsigned kMatchRuns = 12;    // warps with at most this many digit runs rank by match

long long sort_max_tiles_for(long long n) { return (n + kSortTile - 1) / kSortTile; }
long long sort_desc_words(long long max_tiles) {
    return (max_tiles + (max_tiles + kLookBlock - 1) / kLookBlock) * 256;
}

// Digit mask of pass p of a sort over bits [0, end_bit): 8 bits, and end_bit - 8 (passes - 1) bits in
// the last pass (top_mask), so that bits at or above end_bit never take part in the order.
__device__ __forceinline__ unsigned digit_mask(int p, int passes, unsigned top_mask) {
    return p == passes - 1 ? top_mask : 0xffu;
}

__device__ __forceinline__ long long pair_count(const unsigned long long *n_dev, long long n_host, long long cap) {
    long long n = n_dev ? (long long)*(const volatile unsigned long long *)n_dev : n_host;
    return n < cap ? n : cap;
}

// ------------------------------------------------------------------------------------------ histogram
// Adds the digits of keys [0, n) taken by this thread (thread gtid of `stride`) to the per-pass
// shared-memory histograms s_h[pass][256]: four consecutive keys per thread and step, loaded
// before any is counted, so that the lanes of one atomic touch keys four apart (the pairs of one
// Gaussian share their depth bytes: neighbouring keys would collide on one counter).  Keys are
// 16-byte aligned whenever the base is; a misaligned base falls back to single keys.
template <class K>
__device__ __forceinline__ void hist_accumulate(const K *keys, long long n, int passes, unsigned top_mask,
                                                unsigned *s_h, long long gtid, long long stride) {
    constexpr int V = 4;
    const bool vec = ((uintptr_t)keys & 15u) == 0;
    const long long nv = vec ? n / V : 0;
    for (long long c = gtid; c < nv; c += stride) {
        K k[V];
#pragma unroll
        for (int j = 0; j < V; ++j) k[j] = __ldcg(keys + c * V + j);
#pragma unroll
        for (int j = 0; j < V; ++j)
            for (int p = 0; p < passes; ++p)
                atomicAdd(&s_h[p * 256 + ((unsigned)(k[j] >> (8 * p)) & digit_mask(p, passes, top_mask))], 1u);
    }
    for (long long i = nv * V + gtid; i < n; i += stride) {
        const K k = __ldcg(keys + i);
        for (int p = 0; p < passes; ++p)
            atomicAdd(&s_h[p * 256 + ((unsigned)(k >> (8 * p)) & digit_mask(p, passes, top_mask))], 1u);
    }
}

template <class K>
__global__ void __launch_bounds__(512) k_sort_hist(const K *keys, const unsigned long long *n_dev,
                                                   long long n_host, long long cap, int passes, unsigned top_mask,
                                                   unsigned *hist) {
    __shared__ unsigned s_h[8 * 256];
    for (int i = threadIdx.x; i < passes * 256; i += blockDim.x) s_h[i] = 0;
    __syncthreads();
    const long long n = pair_count(n_dev, n_host, cap);
    hist_accumulate(keys, n, passes, top_mask, s_h, (long long)blockIdx.x * blockDim.x + threadIdx.x,
                    (long long)gridDim.x * blockDim.x);
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += blockDim.x)
        if (s_h[i]) atomicAdd(&hist[i], s_h[i]);
}

// One block per pass: exclusive scan of the digit counts; clears the histogram for the next
// sort; block 0 advances the descriptor epoch and resets the scatter tickets.
__global__ void __launch_bounds__(256) k_sort_offsets(unsigned *hist, unsigned *offs, FrameCounters *ctr) {
    __shared__ unsigned s_w[8];
    const int d = threadIdx.x, lane = d & 31, warp = d >> 5;
    const int p = blockIdx.x;
    const unsigned c = hist[p * 256 + d];
    unsigned incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    unsigned wex = 0;
    for (int w = 0; w < warp; ++w) wex += s_w[w];
    offs[p * 256 + d] = wex + incl - c;
    hist[p * 256 + d] = 0;
    if (p == 0 && d == 0) {
        ctr->sort_epoch = ctr->sort_epoch + 1;
        for (int i = 0; i < 8; ++i) ctr->sort_ticket[i] = 0;
    }
}

// ------------------------------------------------------------------------------------------ scatter
// Bulk-copy helpers (the TMA engine's untiled form): one elected thread posts the expected byte
// count on an mbarrier and issues cp.async.bulk copies global -> shared that complete on it.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(unsigned long long *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void bar_expect(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Waits for phase `parity` of the barrier to complete; false after kSpinLimit polls.
__device__ __forceinline__ bool bar_wait(unsigned long long *bar, unsigned parity) {
    for (unsigned it = 0; it < kSpinLimit; ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 32-bit keys (the large tile sorts) double-buffer their tiles so that the next tile's bulk copy
// lands while the current one is scattered; 64-bit keys keep one buffer, so that three CTAs fit
// an SM (their sorts are small and latency-bound).
template <class K>
constexpr int kBufs = sizeof(K) == 4 ? 2 : 1;

// The fused sort of 64-bit keys runs two CTAs per SM with up to 20 items a thread: one wave of
// larger tiles per pass (a room frame's 1.4M pairs in about 300 tiles instead of 460) waits less
// on look-back and barriers than more, smaller tiles (measured: 0.105 vs 0.108 ms; 8 items at 5
// CTAs per SM 0.160 ms).  The per-pass forms keep kMaxItems.
template <class K>
constexpr int kFusedItems = sizeof(K) == 8 ? 20 : kSortItems;
template <class K>
constexpr int kFusedCtas = sizeof(K) == 8 ? 2 : 3;

template <class K, int M = kMaxItems<K>>
struct ScatterSmem {
    K keys[kBufs<K>][kSortThreads * M];   // tile being ranked / next tile in flight
    unsigned vals[kBufs<K>][kSortThreads * M];
    unsigned whist[kSortWarps][256];
    unsigned local_off[256];
    unsigned long long gbase[256];
    unsigned long long bar[2];
    unsigned wsum[kSortWarps];
    long long tile[2];
    int bulk[2];                   // buffer b was filled by a bulk copy (else: plain loads)
};

// Sums the descriptors at entries j, j-1, ..., lo (entry e at base[e * 256]) until one holds an
// inclusive prefix: kLookWindow independent loads per round trip, aggregates added in order, a
// descriptor not yet published re-read after a short sleep.  Returns 1 when a prefix ended the
// walk, 0 when it ran past lo on aggregates alone, 2 on a timeout (status flagged).  The first
// round reads `span` entries.
__device__ __forceinline__ int look_back(const unsigned long long *base, long long j, long long lo,
                                         unsigned long long tag, int span, unsigned &sum, FrameCounters *ctr,
                                         unsigned limit) {
    unsigned spins = 0;
    while (j >= lo) {
        unsigned long long d[kLookWindow];
#pragma unroll
        for (int w = 0; w < kLookWindow; ++w)
            d[w] = (w < span && j - w >= lo) ? *(const volatile unsigned long long *)(base + (j - w) * 256) : 0ull;
        span = kLookWindow;
        int w = 0;
        bool done = false;
#pragma unroll
        for (int q = 0; q < kLookWindow; ++q) {
            if (done || w != q || j - q < lo) continue;
            const unsigned flag = (unsigned)d[q] & ~kDescCount;
            if ((d[q] & 0xffffffff00000000ull) != tag || flag == 0) continue;   // not published yet
            sum += (unsigned)d[q] & kDescCount;
            if (flag == kDescPrefix) done = true;
            w = q + 1;
        }
        if (done) return 1;
        j -= w;
        if (w == 0) {
            if (++spins > limit) {
                atomicOr(&ctr->status, kStTimeout);
                return 2;
            }
            __nanosleep(20);
        }
    }
    return 0;
}

// Starts staging tile t of a pass input into buffer b (one thread): a bulk copy for a full tile of
// 16-byte-aligned 32-bit-key arrays, completing on the buffer's mbarrier; otherwise nothing (the
// tile body loads the tile itself).
template <class K, int M>
__device__ __forceinline__ void stage_tile(ScatterSmem<K, M> &S, int b, long long t, int tsize, const K *kin,
                                           const unsigned *vin, long long nfull, int bulk_ok) {
    S.tile[b] = t;
    const bool bulk = kBufs<K> == 2 && bulk_ok && t < nfull;
    S.bulk[b] = bulk;
    if (bulk) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        bar_expect(&S.bar[b], (unsigned)(tsize * (sizeof(K) + sizeof(unsigned))));
        const int db = kBufs<K> == 2 ? b : 0;
        bulk_g2s(S.keys[db], kin + t * tsize, (unsigned)(tsize * sizeof(K)), &S.bar[b]);
        bulk_g2s(S.vals[db], vin + t * tsize, (unsigned)(tsize * sizeof(unsigned)), &S.bar[b]);
    }
}

// One tile of `items` x 256 pairs (kSortItems <= items <= M, uniform over the CTA) of a
// scatter pass, run by the whole CTA once the per-warp digit counters are zero and the tile's
// staging (stage_tile into buffer b) has been started: load, stable ranking, `publish(cnt)` of
// the tile's count of valid items of digit tid, placement in (digit, rank) order in shared
// memory, `resolve(cnt)` -> the global position of the tile's first item of digit tid, `next()`,
// then the global writes in runs of consecutive addresses.  The onesweep and the
// reduce-then-scan passes differ only in the hooks.  Returns false when the staged copy did not
// arrive (status flagged; uniform over the CTA).
template <class K, int M, class Publish, class Resolve, class Next>
__device__ __forceinline__ bool sort_tile(ScatterSmem<K, M> &S, int b, long long tile, const K *__restrict__ kin,
                                          const unsigned *__restrict__ vin, K *__restrict__ kout,
                                          unsigned *__restrict__ vout, long long n, int items, int shift,
                                          unsigned dmask, FrameCounters *ctr, unsigned &phases, Publish publish,
                                          Resolve resolve,
                                          Next next) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned FULL = 0xffffffffu;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int tsize = kSortThreads * items;
    const int db = kBufs<K> == 2 ? b : 0;      // data buffer of this tile
    const long long tbase = tile * tsize;
    const int wofs = warp * (32 * items);
    bool failed = false;

    K k[M];
    unsigned v[M];
    unsigned rank[(M + 1) / 2] = {};           // two 16-bit in-warp ranks per register
    if (S.bulk[b]) {
        if (bar_wait(&S.bar[b], (phases >> b) & 1u)) {
            phases ^= 1u << b;
        } else {
            if (lane == 0) atomicOr(&ctr->status, kStTimeout);
            failed = true;
        }
#pragma unroll
        for (int i = 0; i < M; ++i) {
            if (i >= items) break;
            k[i] = S.keys[db][wofs + i * 32 + lane];
            v[i] = S.vals[db][wofs + i * 32 + lane];
        }
    } else {
        // L2-only loads: in the fused sort another CTA rewrote these lines since this SM last
        // read them
#pragma unroll
        for (int i = 0; i < M; ++i) {
            if (i >= items) break;
            const long long idx = tbase + wofs + i * 32 + lane;
            if (idx < n) {
                k[i] = __ldcg(kin + idx);
                v[i] = __ldcg(vin + idx);
            } else {
                k[i] = (K)~(K)0;
                v[i] = 0u;
            }
        }
    }
    if (__syncthreads_or(failed)) return false;
    // Per-warp lane masks of each digit, in this tile's value buffer (free until the placement
    // below: the values are in registers).
    unsigned(*mm)[256] = reinterpret_cast<unsigned(*)[256]>(&S.vals[db][0]);
    static_assert(sizeof(S.vals[0]) >= sizeof(unsigned) * kSortWarps * 256, "match masks fit a value buffer");
    for (int i = tid; i < kSortWarps * 256; i += kSortThreads) (&mm[0][0])[i] = 0u;
    __syncthreads();
    // stable warp-level ranking in (item, lane) order
#pragma unroll
    for (int i = 0; i < M; ++i) {
        if (i >= items) break;
        const unsigned d = (unsigned)(k[i] >> shift) & dmask;
        // The lanes holding the same digit: a hardware match costs about as much per distinct
        // value as a shared-memory OR costs per lane colliding on one digit, so the match serves
        // warps whose digits come in few runs (keys of one Gaussian, nearly sorted bytes) and the
        // OR the rest; the run count takes one shuffle and one ballot.
        const unsigned prev = __shfl_up_sync(FULL, d, 1);
        const bool few = __popc(__ballot_sync(FULL, lane == 0 || d != prev)) <= kMatchRuns;
        unsigned peers;
        if (few) {
            peers = __match_any_sync(FULL, d);
        } else {
            atomicOr(&mm[warp][d], 1u << lane);
            __syncwarp();
            peers = mm[warp][d];
        }
        const unsigned before = __popc(peers & lt_mask);
        const unsigned bb = S.whist[warp][d];
        __syncwarp();
        rank[i >> 1] |= (bb + before) << (16 * (i & 1));
        if (before == 0) {
            S.whist[warp][d] = bb + __popc(peers);
            if (!few) mm[warp][d] = 0u;
        }
        __syncwarp();
    }
    __syncthreads();
    // thread tid owns digit tid: warp-exclusive offsets and the tile count
    unsigned cnt = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
        const unsigned c = S.whist[w][tid];
        S.whist[w][tid] = cnt;
        cnt += c;
    }
    // tile-local exclusive scan over digits
    unsigned incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) S.wsum[warp] = incl;
    // the tile's count of valid items for digit tid (padding keys all have the largest digit, dmask,
    // and rank after every valid key of that digit)
    const long long valid_here = min((long long)tsize, n - tbase);
    const unsigned cnt_valid = tid == (int)dmask ? cnt - (unsigned)(tsize - valid_here) : cnt;
    publish(cnt_valid);
    __syncthreads();
    unsigned wex = 0;
    for (int w = 0; w < warp; ++w) wex += S.wsum[w];
    S.local_off[tid] = wex + incl - cnt;
    __syncthreads();
    // place the tile in (digit, rank) order in its own buffer (its contents are in registers)
    // before resolving the global positions, so that no item registers stay live while the
    // onesweep look-back waits
#pragma unroll
    for (int i = 0; i < M; ++i) {
        if (i >= items) break;
        const unsigned d = (unsigned)(k[i] >> shift) & dmask;
        const unsigned pos = S.local_off[d] + S.whist[warp][d] + ((rank[i >> 1] >> (16 * (i & 1))) & 0xffffu);
        S.keys[db][pos] = k[i];
        S.vals[db][pos] = v[i];
    }
    S.gbase[tid] = resolve(cnt_valid);
    next();
    __syncthreads();
    for (int s = tid; s < valid_here; s += kSortThreads) {
        const K key = S.keys[db][s];
        const unsigned d = (unsigned)(key >> shift) & dmask;
        const unsigned long long dst = S.gbase[d] + (unsigned long long)(s - S.local_off[d]);
        kout[dst] = key;
        vout[dst] = S.vals[db][s];
    }
    __syncthreads();
    return true;
}

// The onesweep hooks: publish the tile's count as an aggregate (a prefix for tile 0; a descriptor
// is one self-contained 64-bit word, so nothing it describes needs a fence), and resolve the
// global position by the two-level look-back.  Level 1: the tiles of this block before this one
// (in the first wave every tile has just started, so the whole window is read at once; later a
// tile's predecessor has usually published its prefix, so the first round reads it alone).
// Level 2: whole blocks before this one.  The last tile of a block publishes the block's
// aggregate as soon as level 1 gives it, and the block's prefix with its own.
__device__ __forceinline__ void onesweep_publish(unsigned long long *desc, long long tile, unsigned long long tag,
                                                 unsigned cnt) {
    *(volatile unsigned long long *)(desc + tile * 256 + threadIdx.x) = tag | (tile == 0 ? kDescPrefix : kDescAgg) | cnt;
}

__device__ __forceinline__ unsigned long long onesweep_resolve(unsigned long long *desc, unsigned long long *bdesc,
                                                               long long tile, unsigned long long tag, unsigned goff,
                                                               unsigned cnt, FrameCounters *ctr, unsigned limit) {
    const int tid = threadIdx.x;
    unsigned excl = 0;
    if (tile > 0) {
        static_assert(kLookBlock <= kLookWindow, "one round trip covers a block");
        const long long blk = tile / kLookBlock, lo = blk * kLookBlock;
        const bool last_in_block = tile - lo == kLookBlock - 1;
        int r = look_back(desc + tid, tile - 1, lo, tag, tile < gridDim.x ? kLookWindow : 1, excl, ctr, limit);
        if (r == 0 && blk > 0) {
            if (last_in_block)
                *(volatile unsigned long long *)(bdesc + blk * 256 + tid) = tag | kDescAgg | (excl + cnt);
            r = look_back(bdesc + tid, blk - 1, 0, tag, kLookWindow, excl, ctr, limit);
        }
        (void)r;   // a timeout has flagged the status; the pass's output is then void
        *(volatile unsigned long long *)(desc + tile * 256 + tid) = tag | kDescPrefix | (excl + cnt);
        if (last_in_block)
            *(volatile unsigned long long *)(bdesc + blk * 256 + tid) = tag | kDescPrefix | (excl + cnt);
    }
    return (unsigned long long)goff + excl;
}

// A failed wait leaves copies possibly in flight: give them a bounded chance to land (the phase
// of a buffer is advanced only by a successful wait, so it names the pending one).
template <class K, int M>
__device__ __forceinline__ void drain_staging(ScatterSmem<K, M> &S, unsigned phases) {
    if (threadIdx.x == 0)
        for (int q = 0; q < 2; ++q)
            if (S.bulk[q]) bar_wait(&S.bar[q], (phases >> q) & 1u);
}

// One pass of the onesweep scatter.  Persistent CTAs take tiles in ticket order.  As soon as a
// tile has its global digit offsets (after the look-back), the CTA takes its next ticket and
// starts that tile's bulk copy into the other shared-memory buffer, so the copy overlaps the
// scatter of the current tile (full tiles of 16-byte-aligned arrays; a partial last tile or
// unaligned arrays use plain loads).  Taking the ticket only then keeps a tile's predecessor
// from waiting in a CTA that has not started it.  Progress: every CTA works on its tiles in
// ticket order and a tile waits only on smaller tiles, so the smallest unfinished tile is always
// being worked on.
template <class K>
__global__ void __launch_bounds__(kSortThreads, 3) k_sort_scatter(const K *__restrict__ kin,
                                                               const unsigned *__restrict__ vin,
                                                               K *__restrict__ kout,
                                                               unsigned *__restrict__ vout,
                                                               const unsigned long long *n_dev, long long n_host,
                                                               long long cap, int pass, const unsigned *offs,
                                                               unsigned long long *desc, unsigned long long *bdesc,
                                                               FrameCounters *ctr, int bulk_ok, unsigned limit,
                                                               unsigned dmask) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    ScatterSmem<K> &S = *reinterpret_cast<ScatterSmem<K> *>(smem_raw);
    const int tid = threadIdx.x;
    // an earlier pass gave up waiting: its output is incomplete and this pass's digit offsets
    // (from the first histogram) no longer match it -- write nothing (status already flagged)
    if (__syncthreads_or(tid == 0 && upstream_timed_out(ctr))) return;
    const long long n = pair_count(n_dev, n_host, cap);
    const long long ntiles = (n + kSortTile - 1) / kSortTile;
    const long long nfull = n / kSortTile;
    const unsigned epoch = *(volatile unsigned *)&ctr->sort_epoch;
    const unsigned long long tag = (unsigned long long)(epoch * 8u + (unsigned)pass) << 32;
    const unsigned goff = offs[pass * 256 + tid];
    unsigned phases = 0u;          // bit q: parity of buffer q's next pending phase

    // Takes the next ticket into buffer b and starts its staging.
    auto fetch = [&](int b) {
        if (tid == 0)
            stage_tile(S, b, (long long)atomicAdd(&ctr->sort_ticket[pass], 1u), kSortTile, kin, vin, nfull, bulk_ok);
    };

    if (tid == 0) {
        bar_init(&S.bar[0]);
        bar_init(&S.bar[1]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    fetch(0);
    int b = 0;
    while (true) {
        for (int i = tid; i < kSortWarps * 256; i += kSortThreads) (&S.whist[0][0])[i] = 0;
        __syncthreads();
        const long long tile = S.tile[b];
        if (tile >= ntiles) break;
        // once this tile has published its prefix, take the next ticket, so its copy overlaps
        // the writes while no later tile waits on a ticket that is not being worked on
        if (!sort_tile(
                S, b, tile, kin, vin, kout, vout, n, kSortItems, 8 * pass, dmask, ctr, phases,
                [&](unsigned c) { onesweep_publish(desc, tile, tag, c); },
                [&](unsigned c) { return onesweep_resolve(desc, bdesc, tile, tag, goff, c, ctr, limit); },
                [&] { fetch(b ^ 1); })) {
            drain_staging(S, phases);
            return;
        }
        b ^= 1;
    }
}

template <class K>
static int scatter_grid() {
    static int grid = 0;
    if (grid == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(k_sort_scatter<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(ScatterSmem<K>));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sort_scatter<K>, kSortThreads,
                                                      sizeof(ScatterSmem<K>));
        grid = sms * (per_sm > 0 ? per_sm : 1);
    }
    return grid;
}

// ------------------------------------------------------------------------------------------ fused onesweep
// Grid-wide barrier of a cooperative launch (every CTA resident) on a counter that starts at zero
// and serves this one barrier: after a CTA-wide barrier one thread makes the CTA's writes visible,
// adds its arrival without waiting for the result, and polls until every CTA has arrived.
// Bounded: false after `limit` polls, or as soon as another CTA has flagged a timeout (the
// status then carries kStTimeout).
__device__ __forceinline__ bool grid_barrier(unsigned *count, unsigned ncta, FrameCounters *ctr, unsigned limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        atomicAdd(count, 1u);
        unsigned it = 0;
        while (*(volatile unsigned *)count < ncta) {
            if (++it > limit || (*(volatile unsigned *)&ctr->status & kStTimeout)) {
                atomicOr(&ctr->status, kStTimeout);
                ok = 0;
                break;
            }
            __nanosleep(20);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <class K>
struct FusedSmem {
    ScatterSmem<K, kFusedItems<K>> s;
    unsigned offs[8][256];         // exclusive digit offsets of every pass
};

// The whole sort in one cooperative launch (all CTAs resident, so tiles are dealt statically:
// CTA c takes tiles c, c + G, ...; a tile waits only on smaller tiles, each of which its CTA
// reaches without waiting on larger ones).  The histograms of every pass come first; a grid
// barrier; every CTA scans them into its own digit offsets; then the passes, each ending in a
// grid barrier before the next reads its output.  Removes the per-pass launch gap, the launch
// ramp and the tickets, which dominate sorts of a few thousand tiles.  The pass ping-pongs
// between (k0, v0) and (k1, v1), starting from (k0, v0).  The histograms are cleared for the
// next sort once every CTA has read them (and, after a failed launch, by the frame's counter
// clear); the epoch used for this sort's tags is published for the next one once every CTA has
// read the previous value.  bars: nine counters, zero at the start (barriers 0..7, exits).
template <class K>
__global__ void __launch_bounds__(kSortThreads, kFusedCtas<K>) k_sort_fused(K *k0, unsigned *v0, K *k1, unsigned *v1,
                                                             const unsigned long long *n_dev, long long n_host,
                                                             long long cap, int passes, unsigned *hist,
                                                             unsigned long long *desc, unsigned long long *bdesc,
                                                             FrameCounters *ctr, unsigned *bars, int bulk_ok,
                                                             unsigned limit, unsigned top_mask) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    FusedSmem<K> &F = *reinterpret_cast<FusedSmem<K> *>(smem_raw);
    ScatterSmem<K, kFusedItems<K>> &S = F.s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // an earlier sort of the frame gave up waiting: its output (this sort's input) is incomplete
    if (__syncthreads_or(tid == 0 && upstream_timed_out(ctr))) return;
    const long long n = pair_count(n_dev, n_host, cap);
    // items per thread: the fewest (>= kSortItems) that give every CTA at most one tile, if any do
    int items = kSortItems;
    while (items < kFusedItems<K> && n > (long long)gridDim.x * kSortThreads * items) ++items;
    const int tsize = kSortThreads * items;
    const long long ntiles = (n + tsize - 1) / tsize;
    const long long nfull = n / tsize;
    const unsigned epoch = *(volatile unsigned *)&ctr->sort_epoch + 1u;
    unsigned phases = 0u;
    bool failed = false;

    if (tid == 0) {
        bar_init(&S.bar[0]);
        bar_init(&S.bar[1]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    unsigned *s_h = &S.whist[0][0];
    static_assert(sizeof(S.whist) >= 8 * 256 * sizeof(unsigned), "histograms of 8 passes fit the warp counters");
    for (int i = tid; i < passes * 256; i += kSortThreads) s_h[i] = 0;
    __syncthreads();
    hist_accumulate((const K *)k0, n, passes, top_mask, s_h, (long long)blockIdx.x * kSortThreads + tid,
                    (long long)gridDim.x * kSortThreads);
    __syncthreads();
    for (int i = tid; i < passes * 256; i += kSortThreads)
        if (s_h[i]) atomicAdd(&hist[i], s_h[i]);
    if (!grid_barrier(&bars[0], gridDim.x, ctr, limit)) failed = true;
    if (!failed && blockIdx.x == 0 && tid == 0) atomicMax(&ctr->sort_epoch, epoch);
    unsigned hc[8];
#pragma unroll
    for (int p = 0; p < 8; ++p) hc[p] = p < passes ? __ldcg(hist + p * 256 + tid) : 0u;   // all in flight
#pragma unroll
    for (int p = 0; p < 8; ++p) {
        if (p >= passes || failed) break;
        const unsigned c = hc[p];
        unsigned incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) S.wsum[warp] = incl;
        __syncthreads();
        unsigned wex = 0;
        for (int w = 0; w < warp; ++w) wex += S.wsum[w];
        F.offs[p][tid] = wex + incl - c;
        __syncthreads();
    }
    for (int pass = 0; pass < passes && !failed; ++pass) {
        if (pass == 1 && blockIdx.x == 0)
            for (int i = tid; i < passes * 256; i += kSortThreads) hist[i] = 0u;
        const K *kin = (pass & 1) ? k1 : k0;
        const unsigned *vin = (pass & 1) ? v1 : v0;
        K *kout = (pass & 1) ? k0 : k1;
        unsigned *vout = (pass & 1) ? v0 : v1;
        const unsigned long long tag = (unsigned long long)(epoch * 8u + (unsigned)pass) << 32;
        const unsigned goff = F.offs[pass][tid];
        long long tile = blockIdx.x;
        int b = 0;
        if (tid == 0 && tile < ntiles) {
            // the input was written by other CTAs (generic proxy) before the barrier; the bulk
            // copies read it through the async proxy
            asm volatile("fence.proxy.async.global;" ::: "memory");
            stage_tile(S, b, tile, tsize, kin, vin, nfull, bulk_ok);
        }
        while (tile < ntiles) {
            for (int i = tid; i < kSortWarps * 256; i += kSortThreads) (&S.whist[0][0])[i] = 0;
            __syncthreads();
            const long long nxt = tile + gridDim.x;
            if (!sort_tile(
                    S, b, tile, kin, vin, kout, vout, n, items, 8 * pass, digit_mask(pass, passes, top_mask), ctr,
                    phases,
                    [&](unsigned c) { onesweep_publish(desc, tile, tag, c); },
                    [&](unsigned c) { return onesweep_resolve(desc, bdesc, tile, tag, goff, c, ctr, limit); },
                    [&] {
                        if (tid == 0 && nxt < ntiles) stage_tile(S, b ^ 1, nxt, tsize, kin, vin, nfull, bulk_ok);
                    })) {
                failed = true;
                break;
            }
            tile = nxt;
            b ^= 1;
        }
        if (!failed && pass + 1 < passes && !grid_barrier(&bars[pass + 1], gridDim.x, ctr, limit)) failed = true;
    }
    if (failed) {
        // Some CTAs may have tagged descriptors with this epoch while others gave up before it
        // was published: move the epoch well past every tag this launch can have used.  The
        // barrier counters stay as they are until the frame's counter clear.
        drain_staging(S, phases);
        if (tid == 0) atomicAdd(&ctr->sort_epoch, 1024u);
        return;
    }
    // the last CTA out (every other one has finished its last barrier wait) zeroes the counters
    if (tid == 0 && atomicAdd(&bars[8], 1u) + 1u == gridDim.x)
        for (int i = 0; i <= 8; ++i) *(volatile unsigned *)&bars[i] = 0u;
}

template <class K>
static int fused_grid() {
    static int grid = 0;
    if (grid == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(k_sort_fused<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(FusedSmem<K>));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sort_fused<K>, kSortThreads, sizeof(FusedSmem<K>));
        grid = sms * (per_sm > 0 ? per_sm : 1);
    }
    return grid;
}

// ------------------------------------------------------------------------------------------ reduce-then-scan
// The same stable LSD passes without any inter-CTA waiting: per pass, k_rts_count writes every
// tile's 256 digit counts (digit-major, so that k_rts_scan reads rows), k_rts_scan turns each
// digit's row into exclusive offsets across tiles plus the digit's global offset, and
// k_rts_scatter ranks each tile exactly as the onesweep CTA does and writes it at those offsets.
// It reads the keys twice per pass, but no tile ever waits on a predecessor, so large sorts run at
// the memory system's pace instead of the look-back's.
// Per-tile digit counts, kCountGroup consecutive tiles per CTA step: each tile's keys are loaded
// while the previous tile is counted (plain shared-memory atomics), and thread d writes digit d's
// counts of the group as two 16-byte stores (rows of rts_stride entries, a multiple of
// kCountGroup, so a group never leaves its row).
constexpr int kCountGroup = 8;
template <class K>
__global__ void __launch_bounds__(kSortThreads) k_rts_count(const K *__restrict__ kin, const unsigned long long *n_dev,
                                                            long long n_host, long long cap, int pass,
                                                            unsigned *counts, long long stride,
                                                            const FrameCounters *ctr, unsigned dmask) {
    __shared__ unsigned s_h[kCountGroup][256];
    const int tid = threadIdx.x;
    if (upstream_timed_out(ctr)) return;    // the frame's depth sort gave up: nothing valid to count
    const int shift = 8 * pass;
    const long long n = pair_count(n_dev, n_host, cap);
    const long long ntiles = (n + kSortTile - 1) / kSortTile;
    const long long ngroups = (ntiles + kCountGroup - 1) / kCountGroup;
    auto load = [&](K (&k)[kSortItems], long long tile) {
#pragma unroll
        for (int i = 0; i < kSortItems; ++i) {
            const long long idx = tile * kSortTile + i * kSortThreads + tid;
            k[i] = idx < n ? __ldg(kin + idx) : (K)0;
        }
    };
    for (long long g = blockIdx.x; g < ngroups; g += gridDim.x) {
#pragma unroll
        for (int j = 0; j < kCountGroup; ++j) s_h[j][tid] = 0;
        __syncthreads();
        const long long t0 = g * kCountGroup;
        K nxt[kSortItems];
        load(nxt, t0);
#pragma unroll 1
        for (int j = 0; j < kCountGroup; ++j) {
            K cur[kSortItems];
#pragma unroll
            for (int i = 0; i < kSortItems; ++i) cur[i] = nxt[i];
            if (j + 1 < kCountGroup) load(nxt, t0 + j + 1);
            const long long base = (t0 + j) * kSortTile;
#pragma unroll
            for (int i = 0; i < kSortItems; ++i)
                if (base + i * kSortThreads + tid < n) atomicAdd(&s_h[j][(unsigned)(cur[i] >> shift) & dmask], 1u);
        }
        __syncthreads();
        uint4 *dst = reinterpret_cast<uint4 *>(counts + (long long)tid * stride + t0);
        dst[0] = make_uint4(s_h[0][tid], s_h[1][tid], s_h[2][tid], s_h[3][tid]);
        dst[1] = make_uint4(s_h[4][tid], s_h[5][tid], s_h[6][tid], s_h[7][tid]);
        __syncthreads();
    }
}
static_assert(kCountGroup == 8, "two 16-byte stores per digit and group");

// One CTA per digit: counts[d][t] becomes the sum of counts[d][t'] over t' < t, and the row's total
// goes to tot[d] (the scatter turns the 256 totals into the digits' global offsets).
constexpr int kRtsScanThreads = 1024;
// Row stride of the per-tile digit counts: a multiple of kCountGroup (8), so that every row is
// 32-byte aligned and a count group never leaves its row.
long long rts_stride(long long max_tiles) { return (max_tiles + 7) & ~7ll; }

// One CTA per digit: counts[d][t] becomes the sum of counts[d][t'] over t' < t, and the row's total
// goes to tot[d] (the scatter turns the 256 totals into the digits' global offsets).  The row is
// read and written four entries per thread (16-byte accesses, coalesced), 4096 entries per step,
// with a block-wide scan of the threads' sums and a running carry; entries past the last tile
// count as zero.
__global__ void __launch_bounds__(kRtsScanThreads) k_rts_scan(unsigned *counts, long long stride,
                                                              const unsigned long long *n_dev, long long n_host,
                                                              long long cap, unsigned *tot_out) {
    __shared__ unsigned s_w[kRtsScanThreads / 32];
    const int d = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long n = pair_count(n_dev, n_host, cap);
    const long long ntiles = (n + kSortTile - 1) / kSortTile;
    const long long n4 = (ntiles + 3) / 4;          // within the row: stride is a multiple of 4, >= ntiles
    uint4 *row = reinterpret_cast<uint4 *>(counts + (long long)d * stride);
    unsigned carry = 0;
    for (long long c0 = 0; c0 < n4; c0 += kRtsScanThreads) {
        const long long i = c0 + tid;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (i < n4) {
            v = row[i];
            const long long t = 4 * i;
            if (t + 1 >= ntiles) v.y = 0u;
            if (t + 2 >= ntiles) v.z = 0u;
            if (t + 3 >= ntiles) v.w = 0u;
        }
        const unsigned sum = v.x + v.y + v.z + v.w;
        unsigned incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_w[warp] = incl;
        __syncthreads();
        unsigned wex = 0, tot = 0;
#pragma unroll
        for (int w = 0; w < kRtsScanThreads / 32; ++w) {
            const unsigned x = s_w[w];
            wex += w < warp ? x : 0u;
            tot += x;
        }
        if (i < n4) {
            const unsigned e = carry + wex + incl - sum;
            row[i] = make_uint4(e, e + v.x, e + v.x + v.y, e + v.x + v.y + v.z);
        }
        carry += tot;
        __syncthreads();
    }
    if (tid == 0) tot_out[d] = carry;
}

// Tiles are dealt round-robin, so each CTA knows its next tile: with 32-bit keys its bulk copy
// (full tiles of 16-byte-aligned arrays) lands in the other buffer while this one is ranked.  The
// global position of the tile's first item of digit d is the digit's offset (the exclusive scan
// of the digit totals) plus offs_t[d][tile].
template <class K>
__global__ void __launch_bounds__(kSortThreads, 3) k_rts_scatter(const K *__restrict__ kin,
                                                              const unsigned *__restrict__ vin, K *__restrict__ kout,
                                                              unsigned *__restrict__ vout,
                                                              const unsigned long long *n_dev, long long n_host,
                                                              long long cap, int pass, const unsigned *offs_t,
                                                              long long stride, const unsigned *tot,
                                                              int bulk_ok, FrameCounters *ctr, unsigned dmask) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    ScatterSmem<K> &S = *reinterpret_cast<ScatterSmem<K> *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (__syncthreads_or(tid == 0 && upstream_timed_out(ctr))) return;
    const long long n = pair_count(n_dev, n_host, cap);
    const long long ntiles = (n + kSortTile - 1) / kSortTile;
    const long long nfull = n / kSortTile;
    // global offset of digit tid: exclusive scan of the digit totals
    unsigned dbase;
    {
        const unsigned c = tot[tid];
        unsigned incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) S.wsum[warp] = incl;
        __syncthreads();
        unsigned wex = 0;
        for (int w = 0; w < warp; ++w) wex += S.wsum[w];
        dbase = wex + incl - c;
    }
    unsigned phases = 0u;
    if (tid == 0) {
        bar_init(&S.bar[0]);
        bar_init(&S.bar[1]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0 && blockIdx.x < ntiles) stage_tile(S, 0, (long long)blockIdx.x, kSortTile, kin, vin, nfull, bulk_ok);
    int b = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        for (int i = tid; i < kSortWarps * 256; i += kSortThreads) (&S.whist[0][0])[i] = 0;
        const unsigned long long gb = (unsigned long long)dbase + offs_t[(long long)tid * stride + tile];
        __syncthreads();
        // the other buffer was released at the end of the last tile
        if (tid == 0 && tile + gridDim.x < ntiles)
            stage_tile(S, b ^ 1, tile + gridDim.x, kSortTile, kin, vin, nfull, bulk_ok);
        if (!sort_tile(S, b, tile, kin, vin, kout, vout, n, kSortItems, 8 * pass, dmask, ctr, phases, [](unsigned) {},
                       [&](unsigned) { return gb; }, [] {})) {
            drain_staging(S, phases);
            return;
        }
        b ^= 1;
    }
}

template <class K>
static int rts_scatter_grid() {
    static int grid = 0;
    if (grid == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(k_rts_scatter<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(ScatterSmem<K>));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rts_scatter<K>, kSortThreads, sizeof(ScatterSmem<K>));
        grid = sms * (per_sm > 0 ? per_sm : 1);
    }
    return grid;
}

template <class K>
static int launch_sort_t(K *keys, unsigned *vals, K *keys_tmp, unsigned *vals_tmp, const unsigned long long *n_dev,
                         long long n_host, long long cap, int end_bit, const SortScratch &scr, FrameCounters *ctr,
                         cudaStream_t s) {
    const int passes = (end_bit + 7) / 8;
    const int sgrid = scatter_grid<K>();
    const unsigned limit = wait_limit();
    // the last digit covers bits [8 (passes - 1), end_bit) only
    const unsigned top_mask = (1u << (end_bit - 8 * (passes - 1))) - 1u;
    auto dmask_of = [&](int p) { return p == passes - 1 ? top_mask : 0xffu; };
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long max_tiles = sort_max_tiles_for(cap);
    // full tiles start at multiples of kSortTile elements, so 16-byte-aligned arrays keep every
    // bulk copy 16-byte aligned
    const int bulk_ok = (((uintptr_t)keys | (uintptr_t)vals | (uintptr_t)keys_tmp | (uintptr_t)vals_tmp) & 15u) == 0;
    if (scr.algo == 1 && scr.counts && max_tiles <= scr.max_tiles) {
        const int cgrid = (int)min((long long)sms * 8, max(1ll, (max_tiles + kCountGroup - 1) / kCountGroup));
        const int rgrid = (int)min((long long)rts_scatter_grid<K>(), max_tiles > 0 ? max_tiles : 1);
        K *ka = keys, *kb = keys_tmp;
        unsigned *va = vals, *vb = vals_tmp;
        const long long stride = rts_stride(scr.max_tiles);
        for (int p = 0; p < passes; ++p) {
            k_rts_count<K><<<cgrid, kSortThreads, 0, s>>>(ka, n_dev, n_host, cap, p, scr.counts, stride, ctr,
                                                          dmask_of(p));
            k_rts_scan<<<256, kRtsScanThreads, 0, s>>>(scr.counts, stride, n_dev, n_host, cap, scr.offs + p * 256);
            k_rts_scatter<K><<<rgrid, kSortThreads, sizeof(ScatterSmem<K>), s>>>(ka, va, kb, vb, n_dev, n_host, cap, p,
                                                                               scr.counts, stride,
                                                                               scr.offs + p * 256, bulk_ok, ctr,
                                                                               dmask_of(p));
            K *tk = ka;
            ka = kb;
            kb = tk;
            unsigned *tv = va;
            va = vb;
            vb = tv;
        }
        return passes;
    }
    if (scr.algo == 2 && passes >= 2) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)min((long long)fused_grid<K>(), max_tiles > 0 ? max_tiles : 1));
        cfg.blockDim = dim3(kSortThreads);
        cfg.dynamicSmemBytes = sizeof(FusedSmem<K>);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const cudaError_t e = cudaLaunchKernelEx(&cfg, k_sort_fused<K>, keys, vals, keys_tmp, vals_tmp, n_dev, n_host,
                                                 cap, passes, scr.hist, scr.desc, scr.desc + scr.max_tiles * 256, ctr,
                                                 (unsigned *)((char *)ctr + offsetof(FrameCounters, sort_bar)),
                                                 bulk_ok, limit, top_mask);
        if (e == cudaSuccess) return passes;
        // a cooperative launch refused (e.g. by a device or mode that does not allow it): the
        // error is not sticky, so clear it and run the per-pass form below instead
        cudaGetLastError();
    }
    k_sort_hist<K><<<sms * 2, 512, 0, s>>>(keys, n_dev, n_host, cap, passes, top_mask, scr.hist);
    k_sort_offsets<<<passes, 256, 0, s>>>(scr.hist, scr.offs, ctr);
    int grid = (int)min((long long)sgrid, max_tiles > 0 ? max_tiles : 1);
    K *ka = keys, *kb = keys_tmp;
    unsigned *va = vals, *vb = vals_tmp;
    for (int p = 0; p < passes; ++p) {
        k_sort_scatter<K><<<grid, kSortThreads, sizeof(ScatterSmem<K>), s>>>(ka, va, kb, vb, n_dev, n_host, cap, p,
                                                                             scr.offs, scr.desc,
                                                                             scr.desc + scr.max_tiles * 256, ctr,
                                                                             bulk_ok, limit, dmask_of(p));
        K *tk = ka;
        ka = kb;
        kb = tk;
        unsigned *tv = va;
        va = vb;
        vb = tv;
    }
    return passes;
}

int launch_sort(unsigned long long *keys, unsigned *vals, unsigned long long *keys_tmp, unsigned *vals_tmp,
                const unsigned long long *n_dev, long long n_host, long long cap, int end_bit,
                const SortScratch &scr, FrameCounters *ctr, cudaStream_t s) {
    return launch_sort_t<unsigned long long>(keys, vals, keys_tmp, vals_tmp, n_dev, n_host, cap, end_bit, scr, ctr,
                                             s);
}

int launch_sort32(unsigned *keys, unsigned *vals, unsigned *keys_tmp, unsigned *vals_tmp,
                  const unsigned long long *n_dev, long long cap, int end_bit, const SortScratch &scr,
                  FrameCounters *ctr, cudaStream_t s) {
    return launch_sort_t<unsigned>(keys, vals, keys_tmp, vals_tmp, n_dev, 0, cap, end_bit, scr, ctr, s);
}

// ------------------------------------------------------------------------------------------ ranges
// Key layouts: (tile << 32 | depth bits) as u64 (shift 32), or the tile id alone as u32 (shift 0).
// With at least one and at most kScanPairsPerTile pairs per tile on average, one pass over the
// sorted keys: position i compares the tiles of keys i-1 and i and writes i as the start of every
// tile in between (each start is written once; position n closes the last tiles).  Otherwise a
// binary search per tile.  Grid-stride loops: the grid does not depend on the pair count.
constexpr long long kScanPairsPerTile = 512;
template <class K, int SHIFT>
__global__ void __launch_bounds__(256) k_tile_starts(const K *keys, const unsigned long long *n_dev, long long cap,
                                                     int ntiles, unsigned *starts, const FrameCounters *ctr) {
    if (upstream_timed_out(ctr)) return;    // the sort gave up: its keys may name tiles out of range
    const long long n = pair_count(n_dev, 0, cap);
    const long long g0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (n >= ntiles && n <= kScanPairsPerTile * ntiles) {
        // eight consecutive positions a thread: the keys arrive in 16-byte loads (the key array is
        // 16-byte aligned), plus the key before them
        constexpr int V = 8;
        constexpr int L = V * (int)sizeof(K) / 16;
        for (long long i0 = g0 * V; i0 <= n; i0 += stride * V) {
            K k[V];
            if (i0 + V <= n) {
                const uint4 *src = reinterpret_cast<const uint4 *>(keys + i0);
                uint4 raw[L];
#pragma unroll
                for (int l = 0; l < L; ++l) raw[l] = __ldg(src + l);
                memcpy(k, raw, sizeof(k));
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) k[v] = i0 + v < n ? keys[i0 + v] : (K)0;
            }
            long long prev = i0 == 0 ? -1 : (long long)(keys[i0 - 1] >> SHIFT);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const long long i = i0 + v;
                if (i > n) break;
                const long long cur = i == n ? (long long)ntiles : (long long)(k[v] >> SHIFT);
                for (long long t = prev + 1; t <= cur; ++t) starts[t] = (unsigned)i;
                prev = cur;
            }
        }
        return;
    }
    for (long long b = g0; b <= ntiles; b += stride) {
        const K target = (K)b << SHIFT;
        long long lo = 0, hi = n;
        while (lo < hi) {
            const long long mid = (lo + hi) >> 1;
            if (keys[mid] < target)
                lo = mid + 1;
            else
                hi = mid;
        }
        starts[b] = (unsigned)lo;
    }
}

static int ranges_grid() {
    static int grid = 0;
    if (grid == 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        grid = 8 * sms;
    }
    return grid;
}

void launch_ranges(const unsigned long long *keys, const unsigned long long *n_dev, long long cap, int ntiles,
                   unsigned *starts, const FrameCounters *ctr, cudaStream_t s) {
    k_tile_starts<unsigned long long, 32><<<ranges_grid(), 256, 0, s>>>(keys, n_dev, cap, ntiles, starts, ctr);
}

void launch_ranges32(const unsigned *keys, const unsigned long long *n_dev, long long cap, int ntiles,
                     unsigned *starts, const FrameCounters *ctr, cudaStream_t s) {
    k_tile_starts<unsigned, 0><<<ranges_grid(), 256, 0, s>>>(keys, n_dev, cap, ntiles, starts, ctr);
}

}  // namespace gs
