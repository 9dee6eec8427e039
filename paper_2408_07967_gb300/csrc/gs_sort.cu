// gs_sort.cu -- device-wide LSD radix sort of (u64 key, u32 value) pairs in the onesweep
// form, and the per-tile range search.
//
// Sort (the stage FlashGS inherits from 3DGS's CUB SortPairs, Section 2.2): one pass over the
// keys builds the 256-bin histograms of every 8-bit digit at once; a tiny kernel turns them into
// exclusive digit offsets; then one scatter pass per digit.  A scatter CTA takes tiles of 3072
// pairs in ticket order, ranks them by digit with warp match/ballot (stable: warp-striped load
// order equals input order), publishes its per-digit counts, and reads its predecessors'
// counts through a decoupled look-back over epoch-tagged descriptors (no per-sort clearing;
// waits bounded by kSpinLimit), then scatters through shared memory so that global writes are
// runs of consecutive addresses.
//
// Ranges: the first position of every tile id in the sorted keys by binary search; tile t
// spans [start[t], start[t+1]).
#include "gs_internal.cuh"

namespace gs {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 12;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr unsigned kDescAgg = 1u << 30;
constexpr unsigned kDescPrefix = 2u << 30;
constexpr unsigned kDescCount = (1u << 30) - 1;

int sort_tile_items() { return kSortTile; }
long long sort_max_tiles_for(long long n) { return (n + kSortTile - 1) / kSortTile; }

__device__ __forceinline__ long long pair_count(const unsigned long long *n_dev, long long n_host, long long cap) {
    long long n = n_dev ? (long long)*(const volatile unsigned long long *)n_dev : n_host;
    return n < cap ? n : cap;
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
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
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
template <class K>
struct ScatterSmem {
    K keys[kSortTile];
    unsigned vals[kSortTile];
    unsigned whist[kSortWarps][256];
    unsigned local_off[256];
    unsigned long long gbase[256];
    unsigned wsum[kSortWarps];
    unsigned tile;
};

template <class K>
__global__ void __launch_bounds__(kSortThreads, 3) k_sort_scatter(const K *__restrict__ kin,
                                                               const unsigned *__restrict__ vin,
                                                               K *__restrict__ kout,
                                                               unsigned *__restrict__ vout,
                                                               const unsigned long long *n_dev, long long n_host,
                                                               long long cap, int pass, const unsigned *offs,
                                                               unsigned long long *desc, FrameCounters *ctr) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ScatterSmem<K> &S = *reinterpret_cast<ScatterSmem<K> *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned FULL = 0xffffffffu;
    const int shift = 8 * pass;
    const long long n = pair_count(n_dev, n_host, cap);
    const long long ntiles = (n + kSortTile - 1) / kSortTile;
    const unsigned epoch = *(volatile unsigned *)&ctr->sort_epoch;
    const unsigned long long tag = (unsigned long long)(epoch * 8u + (unsigned)pass) << 32;
    const unsigned lt_mask = (1u << lane) - 1u;
    const unsigned goff = offs[pass * 256 + tid];

    while (true) {
        if (tid == 0) S.tile = atomicAdd(&ctr->sort_ticket[pass], 1u);
        for (int i = tid; i < kSortWarps * 256; i += kSortThreads) (&S.whist[0][0])[i] = 0;
        __syncthreads();
        const long long tile = S.tile;
        if (tile >= ntiles) break;
        const long long tbase = tile * kSortTile;
        const long long wbase = tbase + (long long)warp * (32 * kSortItems);

        K k[kSortItems];
        unsigned v[kSortItems];
        unsigned rank[kSortItems];
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
        // stable warp-level ranking in (item, lane) order
#pragma unroll
        for (int i = 0; i < kSortItems; ++i) {
            const unsigned d = (unsigned)(k[i] >> shift) & 0xffu;
            const unsigned peers = __match_any_sync(FULL, d);
            const unsigned before = __popc(peers & lt_mask);
            const unsigned b = S.whist[warp][d];
            __syncwarp();
            rank[i] = b + before;
            if (before == 0) S.whist[warp][d] = b + __popc(peers);
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
        unsigned long long excl = 0;
        if (tile > 0) {
            long long j = tile - 1;
            unsigned spins = 0;
            while (j >= 0) {
                const unsigned long long d = *(const volatile unsigned long long *)(desc + j * 256 + tid);
                const unsigned flag = (unsigned)d & ~kDescCount;
                if ((d & 0xffffffff00000000ull) != tag || flag == 0) {
                    if (++spins > kSpinLimit) {
                        atomicOr(&ctr->status, kStTimeout);
                        break;
                    }
                    __nanosleep(20);
                    continue;
                }
                excl += (unsigned)d & kDescCount;
                if (flag == kDescPrefix) break;
                --j;
            }
            *(volatile unsigned long long *)my = tag | kDescPrefix | (unsigned)(excl + cnt_valid);
        }
        S.gbase[tid] = (unsigned long long)goff + excl;
        __syncthreads();
        // scatter into shared memory in (digit, rank) order
#pragma unroll
        for (int i = 0; i < kSortItems; ++i) {
            const unsigned d = (unsigned)(k[i] >> shift) & 0xffu;
            const unsigned pos = S.local_off[d] + S.whist[warp][d] + rank[i];
            S.keys[pos] = k[i];
            S.vals[pos] = v[i];
        }
        __syncthreads();
        for (int s = tid; s < valid_here; s += kSortThreads) {
            const K key = S.keys[s];
            const unsigned d = (unsigned)(key >> shift) & 0xffu;
            const unsigned long long dst = S.gbase[d] + (unsigned long long)(s - S.local_off[d]);
            kout[dst] = key;
            vout[dst] = S.vals[s];
        }
        __syncthreads();
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

template <class K>
static int launch_sort_t(K *keys, unsigned *vals, K *keys_tmp, unsigned *vals_tmp, const unsigned long long *n_dev,
                         long long n_host, long long cap, int end_bit, const SortScratch &scr, FrameCounters *ctr,
                         cudaStream_t s) {
    const int passes = (end_bit + 7) / 8;
    const int sgrid = scatter_grid<K>();
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_sort_hist<K><<<sms * 2, 512, 0, s>>>(keys, n_dev, n_host, cap, passes, scr.hist);
    k_sort_offsets<<<passes, 256, 0, s>>>(scr.hist, scr.offs, ctr);
    long long max_tiles = sort_max_tiles_for(cap);
    int grid = (int)min((long long)sgrid, max_tiles > 0 ? max_tiles : 1);
    K *ka = keys, *kb = keys_tmp;
    unsigned *va = vals, *vb = vals_tmp;
    for (int p = 0; p < passes; ++p) {
        k_sort_scatter<K><<<grid, kSortThreads, sizeof(ScatterSmem<K>), s>>>(ka, va, kb, vb, n_dev, n_host, cap, p,
                                                                             scr.offs, scr.desc, ctr);
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
