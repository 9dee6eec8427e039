// gs_sort.cu -- device-wide LSD radix sort of (key, u32 value) pairs in the onesweep form, and
// the per-tile range search.
//
// Sort (the stage FlashGS inherits from 3DGS's CUB SortPairs, Section 2.2): one pass over the
// keys builds the 256-bin histograms of every 8-bit digit at once; a tiny kernel turns them into
// exclusive digit offsets; then one scatter pass per digit.  A scatter CTA takes tiles of 3072
// pairs in ticket order, ranks them by digit with warp match/ballot (stable: warp-striped load
// order equals input order), publishes its per-digit counts, places the tile in (digit, rank)
// order in shared memory, and reads its predecessors' counts through a decoupled look-back over
// epoch-tagged descriptors (no per-sort clearing; waits bounded by kSpinLimit); then it writes runs
// of consecutive addresses.  The look-back has two levels: a tile sums its own block of 16 tiles,
// then whole-block descriptors that the last tile of each block publishes, 16 per round trip, so
// the last of T tiles that all start together waits about 2 + T/256 round trips instead of T/16.
// For 32-bit keys the next tile's keys and values arrive by bulk copy (cp.async.bulk on an
// mbarrier) while the current tile is written out.
//
// Ranges: the first position of every tile id in the sorted keys by binary search; tile t
// spans [start[t], start[t+1]).
#include "gs_internal.cuh"

namespace gs {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 12;
static_assert((kSortThreads * kSortItems * 4) % 16 == 0, "bulk copies of a full tile are whole 16-byte units");
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr unsigned kDescAgg = 1u << 30;
constexpr unsigned kDescPrefix = 2u << 30;
constexpr unsigned kDescCount = (1u << 30) - 1;
constexpr int kLookWindow = 16;        // descriptors per look-back round trip
constexpr int kLookBlock = 16;         // tiles per block descriptor

int sort_tile_items() { return kSortTile; }
long long sort_max_tiles_for(long long n) { return (n + kSortTile - 1) / kSortTile; }
long long sort_desc_words(long long max_tiles) {
    return (max_tiles + (max_tiles + kLookBlock - 1) / kLookBlock) * 256;
}

__device__ __forceinline__ long long pair_count(const unsigned long long *n_dev, long long n_host, long long cap) {
    long long n = n_dev ? (long long)*(const volatile unsigned long long *)n_dev : n_host;
    return n < cap ? n : cap;
}

// Lanes of the warp holding the same 8-bit digit, from eight ballots (one per digit bit): plain
// ALU work at full rate, where a hardware match over 32-bit values is a long-latency operation.
__device__ __forceinline__ unsigned match_digit(unsigned d) {
    unsigned m = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const unsigned bit = (d >> b) & 1u;
        const unsigned bal = __ballot_sync(0xffffffffu, bit);
        m &= bit ? bal : ~bal;
    }
    return m;
}

// ------------------------------------------------------------------------------------------ histogram
template <class K>
__global__ void __launch_bounds__(512) k_sort_hist(const K *keys, const unsigned long long *n_dev,
                                                   long long n_host, long long cap, int passes, unsigned *hist) {
    __shared__ unsigned s_h[8 * 256];
    for (int i = threadIdx.x; i < passes * 256; i += blockDim.x) s_h[i] = 0;
    __syncthreads();
    const long long n = pair_count(n_dev, n_host, cap);
    const long long stride = (long long)gridDim.x * blockDim.x;
    // four keys per thread and step, loaded before any is counted (keys are 16-byte aligned
    // whenever the base is; a misaligned base falls back to single keys)
    constexpr int V = 4;
    const bool vec = ((uintptr_t)keys & 15u) == 0;
    const long long nv = vec ? n / V : 0;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < nv; c += stride) {
        K k[V];
#pragma unroll
        for (int j = 0; j < V; ++j) k[j] = __ldg(keys + c * V + j);
#pragma unroll
        for (int j = 0; j < V; ++j)
            for (int p = 0; p < passes; ++p) atomicAdd(&s_h[p * 256 + (unsigned)((k[j] >> (8 * p)) & 0xffu)], 1u);
    }
    for (long long i = nv * V + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const K k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&s_h[p * 256 + (unsigned)((k >> (8 * p)) & 0xffu)], 1u);
    }
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

template <class K>
struct ScatterSmem {
    K keys[kBufs<K>][kSortTile];   // tile being ranked / next tile in flight
    unsigned vals[kBufs<K>][kSortTile];
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
                                         unsigned long long tag, int span, unsigned &sum, FrameCounters *ctr) {
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
            if (++spins > kSpinLimit) {
                atomicOr(&ctr->status, kStTimeout);
                return 2;
            }
            __nanosleep(20);
        }
    }
    return 0;
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
                                                               FrameCounters *ctr, int bulk_ok) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    ScatterSmem<K> &S = *reinterpret_cast<ScatterSmem<K> *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned FULL = 0xffffffffu;
    const int shift = 8 * pass;
    const long long n = pair_count(n_dev, n_host, cap);
    const long long ntiles = (n + kSortTile - 1) / kSortTile;
    const long long nfull = n / kSortTile;
    const unsigned epoch = *(volatile unsigned *)&ctr->sort_epoch;
    const unsigned long long tag = (unsigned long long)(epoch * 8u + (unsigned)pass) << 32;
    const unsigned lt_mask = (1u << lane) - 1u;
    const unsigned goff = offs[pass * 256 + tid];
    unsigned phases = 0u;          // bit q: parity of buffer q's next pending phase
    bool failed = false;

    // Takes the next ticket into buffer b and starts its bulk copy when it is a full tile.
    auto fetch = [&](int b) {
        if (tid == 0) {
            const long long t = (long long)atomicAdd(&ctr->sort_ticket[pass], 1u);
            S.tile[b] = t;
            const bool bulk = kBufs<K> == 2 && bulk_ok && t < nfull;
            S.bulk[b] = bulk;
            if (bulk) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                bar_expect(&S.bar[b], (unsigned)(kSortTile * (sizeof(K) + sizeof(unsigned))));
                const int db = kBufs<K> == 2 ? b : 0;
                bulk_g2s(S.keys[db], kin + t * kSortTile, (unsigned)(kSortTile * sizeof(K)), &S.bar[b]);
                bulk_g2s(S.vals[db], vin + t * kSortTile, (unsigned)(kSortTile * sizeof(unsigned)), &S.bar[b]);
            }
        }
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
        const int db = kBufs<K> == 2 ? b : 0;      // data buffer of this tile
        const long long tbase = tile * kSortTile;
        const int wofs = warp * (32 * kSortItems);

        K k[kSortItems];
        unsigned v[kSortItems];
        unsigned rank[kSortItems];
        if (S.bulk[b]) {
            if (bar_wait(&S.bar[b], (phases >> b) & 1u)) {
                phases ^= 1u << b;
            } else {
                if (lane == 0) atomicOr(&ctr->status, kStTimeout);
                failed = true;
            }
#pragma unroll
            for (int i = 0; i < kSortItems; ++i) {
                k[i] = S.keys[db][wofs + i * 32 + lane];
                v[i] = S.vals[db][wofs + i * 32 + lane];
            }
        } else {
#pragma unroll
            for (int i = 0; i < kSortItems; ++i) {
                const long long idx = tbase + wofs + i * 32 + lane;
                if (idx < n) {
                    k[i] = kin[idx];
                    v[i] = vin[idx];
                } else {
                    k[i] = (K)~(K)0;
                    v[i] = 0u;
                }
            }
        }
        if (__syncthreads_or(failed)) break;
        // stable warp-level ranking in (item, lane) order
#pragma unroll
        for (int i = 0; i < kSortItems; ++i) {
            const unsigned d = (unsigned)(k[i] >> shift) & 0xffu;
            const unsigned peers = __match_any_sync(FULL, d);   // latency: it precedes the publish
            const unsigned before = __popc(peers & lt_mask);
            const unsigned bb = S.whist[warp][d];
            __syncwarp();
            rank[i] = bb + before;
            if (before == 0) S.whist[warp][d] = bb + __popc(peers);
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
        // publish this tile's count of valid items for digit tid, then look back
        const long long valid_here = min((long long)kSortTile, n - tbase);
        const unsigned cnt_valid = tid == 255 ? cnt - (unsigned)(kSortTile - valid_here) : cnt;
        unsigned long long *my = desc + tile * 256 + tid;
        __threadfence();
        if (tile == 0) {
            *(volatile unsigned long long *)my = tag | kDescPrefix | cnt_valid;
        } else {
            *(volatile unsigned long long *)my = tag | kDescAgg | cnt_valid;
        }
        __syncthreads();
        unsigned wex = 0;
        for (int w = 0; w < warp; ++w) wex += S.wsum[w];
        S.local_off[tid] = wex + incl - cnt;
        __syncthreads();
        // scatter into this tile's buffer (its contents are in registers) in (digit, rank) order
        // before the look-back, so that only the digit's registers stay live while it waits
#pragma unroll
        for (int i = 0; i < kSortItems; ++i) {
            const unsigned d = (unsigned)(k[i] >> shift) & 0xffu;
            const unsigned pos = S.local_off[d] + S.whist[warp][d] + rank[i];
            S.keys[db][pos] = k[i];
            S.vals[db][pos] = v[i];
        }
        unsigned excl = 0;
        if (tile > 0) {
            // Level 1: the tiles of this block before this one (in the first wave every tile has
            // just started, so the whole window is read at once; later a tile's predecessor has
            // usually published its prefix, so the first round reads it alone).  Level 2: whole
            // blocks before this one.  The last tile of a block publishes the block's aggregate
            // as soon as level 1 gives it, and the block's prefix with its own.
            static_assert(kLookBlock <= kLookWindow, "one round trip covers a block");
            const long long blk = tile / kLookBlock, lo = blk * kLookBlock;
            const bool last_in_block = tile - lo == kLookBlock - 1;
            int r = look_back(desc + tid, tile - 1, lo, tag, tile < gridDim.x ? kLookWindow : 1, excl, ctr);
            if (r == 0 && blk > 0) {
                if (last_in_block)
                    *(volatile unsigned long long *)(bdesc + blk * 256 + tid) = tag | kDescAgg | (excl + cnt_valid);
                r = look_back(bdesc + tid, blk - 1, 0, tag, kLookWindow, excl, ctr);
            }
            (void)r;   // a timeout has flagged the status; the pass's output is then void
            *(volatile unsigned long long *)my = tag | kDescPrefix | (excl + cnt_valid);
            if (last_in_block)
                *(volatile unsigned long long *)(bdesc + blk * 256 + tid) = tag | kDescPrefix | (excl + cnt_valid);
        }
        S.gbase[tid] = (unsigned long long)goff + excl;
        // this tile has published its prefix: take the next ticket now, so its copy overlaps the
        // scatter below while no later tile waits on a ticket that is not being worked on
        fetch(b ^ 1);
        __syncthreads();
        for (int s = tid; s < valid_here; s += kSortThreads) {
            const K key = S.keys[db][s];
            const unsigned d = (unsigned)(key >> shift) & 0xffu;
            const unsigned long long dst = S.gbase[d] + (unsigned long long)(s - S.local_off[d]);
            kout[dst] = key;
            vout[dst] = S.vals[db][s];
        }
        __syncthreads();
        b ^= 1;
    }
    // a failed wait leaves copies possibly in flight: give them a bounded chance to land (the
    // phase of a buffer is advanced only by a successful wait, so it names the pending one)
    if (failed && tid == 0) {
        for (int q = 0; q < 2; ++q)
            if (S.bulk[q]) bar_wait(&S.bar[q], (phases >> q) & 1u);
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

// ------------------------------------------------------------------------------------------ reduce-then-scan
// The same stable LSD passes without any inter-CTA waiting: per pass, k_rts_count writes every
// tile's 256 digit counts (digit-major, so that k_rts_scan reads rows), k_rts_scan turns each
// digit's row into exclusive offsets across tiles plus the digit's global offset, and
// k_rts_scatter ranks each tile exactly as the onesweep CTA does and writes it at those offsets.
// It reads the keys twice per pass, but no tile ever waits on a predecessor, so large sorts run at
// the memory system's pace instead of the look-back's.
template <class K>
__global__ void __launch_bounds__(kSortThreads) k_rts_count(const K *__restrict__ kin, const unsigned long long *n_dev,
                                                            long long n_host, long long cap, int pass,
                                                            unsigned *counts, long long stride) {
    __shared__ unsigned s_h[256];
    const int tid = threadIdx.x, lane = tid & 31;
    const int shift = 8 * pass;
    const long long n = pair_count(n_dev, n_host, cap);
    const long long ntiles = (n + kSortTile - 1) / kSortTile;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        s_h[tid] = 0;
        __syncthreads();
        const long long base = tile * kSortTile;
        unsigned dg[kSortItems];
#pragma unroll
        for (int i = 0; i < kSortItems; ++i) {        // all loads in flight before any ranking
            const long long idx = base + i * kSortThreads + tid;
            dg[i] = idx < n ? (unsigned)(__ldg(kin + idx) >> shift) & 0xffu : 256u;
        }
#pragma unroll
        for (int i = 0; i < kSortItems; ++i)
            if (dg[i] < 256u) atomicAdd(&s_h[dg[i]], 1u);
        __syncthreads();
        counts[(long long)tid * stride + tile] = s_h[tid];
        __syncthreads();
    }
}

// One CTA per digit: counts[d][t] becomes the sum of counts[d][t'] over t' < t, and the row's total
// goes to tot[d] (the scatter turns the 256 totals into the digits' global offsets).
constexpr int kRtsScanThreads = 1024;
constexpr int kRtsScanRun = 24;   // 24576 tiles per sweep
__global__ void __launch_bounds__(kRtsScanThreads) k_rts_scan(unsigned *counts, long long stride,
                                                              const unsigned long long *n_dev, long long n_host,
                                                              long long cap, unsigned *tot_out) {
    __shared__ unsigned s_w[kRtsScanThreads / 32];
    __shared__ unsigned s_carry;
    const int d = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long n = pair_count(n_dev, n_host, cap);
    const long long ntiles = (n + kSortTile - 1) / kSortTile;
    unsigned *row = counts + (long long)d * stride;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (long long b0 = 0; b0 < ntiles; b0 += (long long)kRtsScanThreads * kRtsScanRun) {
        const long long my0 = b0 + (long long)tid * kRtsScanRun;
        unsigned sum = 0;
#pragma unroll 8
        for (int r = 0; r < kRtsScanRun; ++r)
            if (my0 + r < ntiles) sum += row[my0 + r];
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
        unsigned run = s_carry + wex + incl - sum;
#pragma unroll 8
        for (int r = 0; r < kRtsScanRun; ++r)
            if (my0 + r < ntiles) {
                const unsigned x = row[my0 + r];    // read before this thread overwrites it
                row[my0 + r] = run;
                run += x;
            }
        __syncthreads();
        if (tid == 0) s_carry += tot;
        __syncthreads();
    }
    if (tid == 0) tot_out[d] = s_carry;
}

template <class K>
struct RtsSmem {
    K keys[kBufs<K>][kSortTile];     // tile being ranked / next tile arriving (32-bit keys)
    unsigned vals[kBufs<K>][kSortTile];
    unsigned whist[kSortWarps][256];
    unsigned local_off[256];
    unsigned gbase[256];
    unsigned wsum[kSortWarps];
    unsigned long long bar[2];
};

template <class K>
__global__ void __launch_bounds__(kSortThreads, 3) k_rts_scatter(const K *__restrict__ kin,
                                                              const unsigned *__restrict__ vin, K *__restrict__ kout,
                                                              unsigned *__restrict__ vout,
                                                              const unsigned long long *n_dev, long long n_host,
                                                              long long cap, int pass, const unsigned *offs_t,
                                                              long long stride, const unsigned *tot,
                                                              int bulk_ok, FrameCounters *ctr) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    RtsSmem<K> &S = *reinterpret_cast<RtsSmem<K> *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned FULL = 0xffffffffu;
    const int shift = 8 * pass;
    const long long n = pair_count(n_dev, n_host, cap);
    const long long ntiles = (n + kSortTile - 1) / kSortTile;
    const unsigned lt_mask = (1u << lane) - 1u;
    // global offset of digit tid: exclusive scan of the digit totals
    unsigned dbase;
    {
        const unsigned c = tot[tid];
        unsigned incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) S.wsum[warp] = incl;
        __syncthreads();
        unsigned wex = 0;
        for (int w = 0; w < warp; ++w) wex += S.wsum[w];
        dbase = wex + incl - c;
        __syncthreads();
    }
    // Tiles are dealt round-robin, so each CTA knows its next tile: with 32-bit keys its bulk copy
    // (full tiles of 16-byte-aligned arrays) lands in the other buffer while this one is ranked.
    const long long nfull = n / kSortTile;
    constexpr bool kPrefetch = kBufs<K> == 2;
    unsigned phases = 0u;
    bool failed = false;
    auto issue = [&](long long t, int b) {
        if (kPrefetch && tid == 0 && bulk_ok && t < nfull) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            bar_expect(&S.bar[b], (unsigned)(kSortTile * (sizeof(K) + sizeof(unsigned))));
            bulk_g2s(S.keys[b], kin + t * kSortTile, (unsigned)(kSortTile * sizeof(K)), &S.bar[b]);
            bulk_g2s(S.vals[b], vin + t * kSortTile, (unsigned)(kSortTile * sizeof(unsigned)), &S.bar[b]);
        }
    };
    if (kPrefetch && tid == 0) {
        bar_init(&S.bar[0]);
        bar_init(&S.bar[1]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    issue(blockIdx.x, 0);
    int it = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int b = kPrefetch ? (it & 1) : 0;
        for (int i = tid; i < kSortWarps * 256; i += kSortThreads) (&S.whist[0][0])[i] = 0;
        S.gbase[tid] = dbase + offs_t[(long long)tid * stride + tile];
        issue(tile + gridDim.x, b ^ 1);      // the other buffer was released at the end of the last tile
        const long long tbase = tile * kSortTile;
        const long long wbase = tbase + (long long)warp * (32 * kSortItems);
        K k[kSortItems];
        unsigned v[kSortItems];
        unsigned rank[kSortItems];
        if (kPrefetch && bulk_ok && tile < nfull) {
            if (bar_wait(&S.bar[b], (phases >> b) & 1u)) {
                phases ^= 1u << b;
            } else {
                if (lane == 0) atomicOr(&ctr->status, kStTimeout);
                failed = true;
            }
            const int wofs = warp * (32 * kSortItems);
#pragma unroll
            for (int i = 0; i < kSortItems; ++i) {
                k[i] = S.keys[b][wofs + i * 32 + lane];
                v[i] = S.vals[b][wofs + i * 32 + lane];
            }
        } else {
#pragma unroll
            for (int i = 0; i < kSortItems; ++i) {
                const long long idx = wbase + i * 32 + lane;
                if (idx < n) {
                    k[i] = kin[idx];
                    v[i] = vin[idx];
                } else {
                    k[i] = (K)~(K)0;
                    v[i] = 0u;
                }
            }
        }
        if (__syncthreads_or(failed)) break;
#pragma unroll
        for (int i = 0; i < kSortItems; ++i) {
            const unsigned d = (unsigned)(k[i] >> shift) & 0xffu;
            const unsigned peers = match_digit(d);
            const unsigned before = __popc(peers & lt_mask);
            const unsigned bb = S.whist[warp][d];
            __syncwarp();
            rank[i] = bb + before;
            if (before == 0) S.whist[warp][d] = bb + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        unsigned cnt = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            const unsigned c = S.whist[w][tid];
            S.whist[w][tid] = cnt;
            cnt += c;
        }
        unsigned incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) S.wsum[warp] = incl;
        __syncthreads();
        unsigned wex = 0;
        for (int w = 0; w < warp; ++w) wex += S.wsum[w];
        S.local_off[tid] = wex + incl - cnt;
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kSortItems; ++i) {
            const unsigned d = (unsigned)(k[i] >> shift) & 0xffu;
            const unsigned pos = S.local_off[d] + S.whist[warp][d] + rank[i];
            S.keys[b][pos] = k[i];
            S.vals[b][pos] = v[i];
        }
        __syncthreads();
        const long long valid_here = min((long long)kSortTile, n - tbase);
        for (int s = tid; s < valid_here; s += kSortThreads) {
            const K key = S.keys[b][s];
            const unsigned d = (unsigned)(key >> shift) & 0xffu;
            const unsigned long long dst = (unsigned long long)S.gbase[d] + (unsigned long long)(s - S.local_off[d]);
            kout[dst] = key;
            vout[dst] = S.vals[b][s];
        }
        __syncthreads();
    }
    // a failed wait leaves copies possibly in flight: give them a bounded chance to land
    if (kPrefetch && failed && tid == 0) {
        bar_wait(&S.bar[0], phases & 1u);
        bar_wait(&S.bar[1], (phases >> 1) & 1u);
    }
}

template <class K>
static int rts_scatter_grid() {
    static int grid = 0;
    if (grid == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(k_rts_scatter<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(RtsSmem<K>));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rts_scatter<K>, kSortThreads, sizeof(RtsSmem<K>));
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
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long max_tiles = sort_max_tiles_for(cap);
    // full tiles start at multiples of kSortTile elements, so 16-byte-aligned arrays keep every
    // bulk copy 16-byte aligned
    const int bulk_ok = (((uintptr_t)keys | (uintptr_t)vals | (uintptr_t)keys_tmp | (uintptr_t)vals_tmp) & 15u) == 0;
    if (scr.algo == 1 && scr.counts && max_tiles <= scr.max_tiles) {
        const int cgrid = (int)min((long long)sms * 8, max_tiles > 0 ? max_tiles : 1);
        const int rgrid = (int)min((long long)rts_scatter_grid<K>(), max_tiles > 0 ? max_tiles : 1);
        K *ka = keys, *kb = keys_tmp;
        unsigned *va = vals, *vb = vals_tmp;
        for (int p = 0; p < passes; ++p) {
            k_rts_count<K><<<cgrid, kSortThreads, 0, s>>>(ka, n_dev, n_host, cap, p, scr.counts, scr.max_tiles);
            k_rts_scan<<<256, kRtsScanThreads, 0, s>>>(scr.counts, scr.max_tiles, n_dev, n_host, cap,
                                                       scr.offs + p * 256);
            k_rts_scatter<K><<<rgrid, kSortThreads, sizeof(RtsSmem<K>), s>>>(ka, va, kb, vb, n_dev, n_host, cap, p,
                                                                           scr.counts, scr.max_tiles,
                                                                           scr.offs + p * 256, bulk_ok, ctr);
            K *tk = ka;
            ka = kb;
            kb = tk;
            unsigned *tv = va;
            va = vb;
            vb = tv;
        }
        return passes;
    }
    k_sort_hist<K><<<sms * 2, 512, 0, s>>>(keys, n_dev, n_host, cap, passes, scr.hist);
    k_sort_offsets<<<passes, 256, 0, s>>>(scr.hist, scr.offs, ctr);
    int grid = (int)min((long long)sgrid, max_tiles > 0 ? max_tiles : 1);
    K *ka = keys, *kb = keys_tmp;
    unsigned *va = vals, *vb = vals_tmp;
    for (int p = 0; p < passes; ++p) {
        k_sort_scatter<K><<<grid, kSortThreads, sizeof(ScatterSmem<K>), s>>>(ka, va, kb, vb, n_dev, n_host, cap, p,
                                                                             scr.offs, scr.desc,
                                                                             scr.desc + scr.max_tiles * 256, ctr,
                                                                             bulk_ok);
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
template <class K, int SHIFT>
__global__ void k_tile_starts(const K *keys, const unsigned long long *n_dev, long long cap, int ntiles,
                              unsigned *starts) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > ntiles) return;
    const long long n = pair_count(n_dev, 0, cap);
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

void launch_ranges(const unsigned long long *keys, const unsigned long long *n_dev, long long cap, int ntiles,
                   unsigned *starts, cudaStream_t s) {
    const int threads = 256;
    const int blocks = (ntiles + 1 + threads - 1) / threads;
    k_tile_starts<unsigned long long, 32><<<blocks, threads, 0, s>>>(keys, n_dev, cap, ntiles, starts);
}

void launch_ranges32(const unsigned *keys, const unsigned long long *n_dev, long long cap, int ntiles,
                     unsigned *starts, cudaStream_t s) {
    const int threads = 256;
    const int blocks = (ntiles + 1 + threads - 1) / threads;
    k_tile_starts<unsigned, 0><<<blocks, threads, 0, s>>>(keys, n_dev, cap, ntiles, starts);
}

}  // namespace gs
