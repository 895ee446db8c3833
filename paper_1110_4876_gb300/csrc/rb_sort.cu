// rb_sort.cu -- stable LSD radix sort of (64-bit key, 32-bit value) pairs and
// an exclusive scan of int32 arrays, both sized on the device.
//
// The sort replaces the insertion/reconstruction of the paper's tree
// (Sect. 4.2): particles are put in Morton order so that every cell is a
// contiguous range.  One launch counts the digits of every pass; then each
// 8-bit digit pass is one launch that ranks keys within a tile with warp
// ballots and finds the tile's place among the earlier tiles by a
// bounded decoupled look-back over per-tile status words.
#include "rb_internal.cuh"

namespace rb {

namespace {
constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;   // 2048 keys per block
constexpr int kBins = 256;
constexpr int kScanThreads = 1024;

__device__ __forceinline__ int read_n(const int* d_n, int ncap) {
    if (!d_n) return ncap;
    int n = *d_n;
    return n < ncap ? n : ncap;
}

// Status words of the decoupled look-back: a tile's count of one digit with
// a two-bit flag (0: not yet published, aggregate: this tile's own count,
// prefix: this tile's count plus every earlier tile's).  Flag and count
// share one 32-bit word, so a single store publishes both.
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagPre = 2u << 30;
constexpr uint32_t kCountMask = (1u << 30) - 1u;
constexpr int kMaxPasses = 12;   // 64-bit keys: 8 digits; 32-bit box digits: 4
constexpr int kLook = 16;   // predecessors read per look-back step
constexpr unsigned long long kLookLimitNs = 500000000ull;   // half a second

__device__ __forceinline__ unsigned long long sort_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The lanes of act whose 8-bit digit equals this lane's: one ballot per
// digit bit (a match-any vote through eight ballots; a pass with them took
// 21 us at 1M keys against 23 us with the match instruction).  Every lane of
// the warp must call it.
__device__ __forceinline__ unsigned digit_peers(unsigned act, uint32_t d) {
    unsigned peers = act;
#pragma unroll
    for (int b = 0; b < 8; b++) {
        const bool bit = (d >> b) & 1u;
        const unsigned m = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? m : ~m;
    }
    return peers;
}

// Digit counts of every pass in one read of the keys (the digit multiset of
// a pass does not depend on the order the earlier passes leave), plus the
// zeroing of both status banks for the tiles in use.  A thread counts
// kItems consecutive keys and adds each run of equal digits with one shared
// atomic: nearly sorted keys share their high digits over long runs.
// hist[p * 256 + d] must be zero on entry (the caller clears it).
template <bool kHasBox>
__global__ void __launch_bounds__(kThreads) k_rs_hist(const uint64_t* __restrict__ key,
                                                      const uint32_t* __restrict__ val,
                                                      const int32_t* __restrict__ box,
                                                      const int* d_n, int ncap, int passes_key,
                                                      int passes_box, uint32_t* __restrict__ hist,
                                                      uint32_t* __restrict__ status, int tiles_cap) {
    __shared__ uint32_t h[kMaxPasses][kBins];
    const int P = passes_key + passes_box;
    for (int i = threadIdx.x; i < P * kBins; i += kThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    const int n = read_n(d_n, ncap);
    const int nt = (n + kTile - 1) / kTile;
    const size_t rows = (size_t)nt * kBins;
    const size_t stride = (size_t)gridDim.x * kThreads;
    for (size_t w = (size_t)blockIdx.x * kThreads + threadIdx.x; w < 2 * rows; w += stride) {
        const size_t bank = w >= rows ? 1 : 0;
        status[bank * (size_t)tiles_cap * kBins + (w - bank * rows)] = 0u;
    }
    for (long long i0 = ((long long)blockIdx.x * kThreads + threadIdx.x) * kItems; i0 < n;
         i0 += (long long)stride * kItems) {
        const int c = (int)min((long long)kItems, (long long)n - i0);
        uint64_t k[kItems];
        uint32_t bd[kItems];
#pragma unroll
        for (int r = 0; r < kItems; r++) {
            k[r] = r < c ? key[i0 + r] : 0ull;
            bd[r] = kHasBox && r < c ? (uint32_t)box[val[i0 + r]] : 0u;
        }
        for (int p = 0; p < P; p++) {
            const bool bp = kHasBox && p >= passes_key;
            const int sh = bp ? 8 * (p - passes_key) : 8 * p;
            uint32_t run_d = bp ? (bd[0] >> sh) & 255u : (uint32_t)(k[0] >> sh) & 255u;
            uint32_t run_c = 1;
#pragma unroll
            for (int r = 1; r < kItems; r++) {
                if (r < c) {
                    const uint32_t dg = bp ? (bd[r] >> sh) & 255u : (uint32_t)(k[r] >> sh) & 255u;
                    if (dg == run_d) {
                        run_c++;
                    } else {
                        atomicAdd(&h[p][run_d], run_c);
                        run_d = dg;
                        run_c = 1;
                    }
                }
            }
            atomicAdd(&h[p][run_d], run_c);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < P * kBins; i += kThreads) {
        const uint32_t c = (&h[0][0])[i];
        if (c) atomicAdd(&hist[i], c);
    }
}

// Exclusive scan of `total` words in place by one block; the sum of all
// words goes to *sum when sum is non-null.
template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_block(T* __restrict__ a, int total,
                                                             T* __restrict__ sum) {
    __shared__ T warp_sums[kScanThreads / 32];
    const int per = (total + kScanThreads - 1) / kScanThreads;
    const int b = threadIdx.x * per;
    const int e = min(b + per, total);
    T s = 0;
    for (int i = b; i < e; i++) s += a[i];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T v = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) warp_sums[w] = v;
    __syncthreads();
    if (w == 0) {
        T x = warp_sums[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        warp_sums[lane] = x;
    }
    __syncthreads();
    T run = v - s + (w > 0 ? warp_sums[w - 1] : T(0));
    for (int i = b; i < e; i++) {
        T c = a[i];
        a[i] = run;
        run += c;
    }
    if (sum && threadIdx.x == kScanThreads - 1) *sum = run;
}

// One digit pass, one launch: block b takes tile b (2048 keys).  It ranks
// the tile's keys with warp ballots, publishes its per-digit counts, finds
// the counts of all earlier tiles by looking back over their status words
// (decoupled look-back: sum aggregates until a prefix is met), and writes
// the tile in digit order.  A tile waits only on smaller tiles, whose blocks
// the GPU dispatched before it (blocks start in index order) and which
// publish before they wait themselves, so the waits end whether or not the
// whole grid is resident, also beside other kernels; each wait is bounded
// all the same (half a second, or at once when another wait gave up) and
// reports kErrSortStall when it gives up.  Stable: within a tile keys keep
// their order, and the tiles are in key order.
template <bool kBoxDigit>
__global__ void __launch_bounds__(kThreads, 4) k_rs_pass(const uint64_t* __restrict__ kin,
                                                      const uint32_t* __restrict__ vin,
                                                      uint64_t* __restrict__ kout,
                                                      uint32_t* __restrict__ vout,
                                                      const int32_t* __restrict__ box,
                                                      const int* d_n, int ncap, int shift, int pass,
                                                      const uint32_t* __restrict__ hist,
                                                      uint32_t* __restrict__ status, int tiles_cap,
                                                      int* __restrict__ err) {
    __shared__ uint32_t wcnt[kThreads / 32][kBins];
    __shared__ uint32_t gstart[kBins];   // where digit d of this tile starts in the output
    __shared__ uint32_t lstart[kBins];   // where digit d starts inside the tile
    __shared__ uint32_t wsum[kThreads / 32];
    __shared__ uint64_t sk[kTile];
    __shared__ uint32_t sv[kTile];
    const int n = read_n(d_n, ncap);
    if ((long long)blockIdx.x * kTile >= n) return;   // past the keys in use
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int d = threadIdx.x;   // the digit this thread counts and looks back for
    uint32_t* mine = status + (size_t)(pass & 1) * tiles_cap * kBins;
    uint32_t* other = status + (size_t)((pass & 1) ^ 1) * tiles_cap * kBins;
    uint32_t digit_base;
    {
        // exclusive scan of this pass's digit totals: where digit d starts
        const uint32_t tot = hist[pass * kBins + d];
        uint32_t v = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        if (lane == 31) wsum[warp] = v;
        __syncthreads();
        uint32_t before = 0;
        for (int w = 0; w < warp; w++) before += wsum[w];
        digit_base = before + v - tot;
    }
    const unsigned lt = (1u << lane) - 1u;
    const int tile = blockIdx.x;
    if (tile * kTile < n) {
        const int base = tile * kTile;
        const int tn = min(kTile, n - base);
        // the other bank held the previous pass's words; clear this tile's
        // row of it for the next pass
        other[(size_t)tile * kBins + d] = 0u;
        for (int q = threadIdx.x; q < (kThreads / 32) * kBins; q += kThreads) (&wcnt[0][0])[q] = 0;
        __syncthreads();
        uint64_t k[kItems];
        uint32_t v[kItems];
        uint32_t pos[kItems];
        int dig[kItems];
        const int wbase = base + warp * (kTile / (kThreads / 32));
        // all loads first: the ranking below orders shared-memory updates
        // with __syncwarp, which would otherwise keep each item's loads
        // behind the previous item's
#pragma unroll
        for (int r = 0; r < kItems; r++) {
            const int i = wbase + r * 32 + lane;
            const bool ok = i < n;
            k[r] = ok ? kin[i] : 0ull;
            v[r] = ok ? vin[i] : 0u;
        }
#pragma unroll
        for (int r = 0; r < kItems; r++) {
            const bool ok = wbase + r * 32 + lane < n;
            int dd = 0;
            if (ok) dd = kBoxDigit ? (int)((box[v[r]] >> shift) & 255) : (int)((k[r] >> shift) & 255ull);
            dig[r] = ok ? dd : -1;
        }
#pragma unroll
        for (int r = 0; r < kItems; r++) {
            const bool ok = dig[r] >= 0;
            const int dd = ok ? dig[r] : 0;
            const unsigned act = __ballot_sync(0xffffffffu, ok);
            const unsigned peers = digit_peers(act, (uint32_t)dd);
            pos[r] = 0;
            if (ok) {
                const int rank = __popc(peers & lt);
                const uint32_t c = wcnt[warp][dd];
                pos[r] = c + rank;
                __syncwarp(act);
                if (rank == 0) wcnt[warp][dd] = c + __popc(peers);
                __syncwarp(act);
            }
        }
        __syncthreads();
        uint32_t cnt = 0;   // this tile's keys of digit d
#pragma unroll
        for (int w = 0; w < kThreads / 32; w++) {
            const uint32_t x = wcnt[w][d];
            wcnt[w][d] = cnt;
            cnt += x;
        }
        volatile uint32_t* row = mine + (size_t)tile * kBins;
        row[d] = (tile == 0 ? kFlagPre : kFlagAgg) | cnt;
        {
            // where digit d starts inside the tile (block scan of the counts)
            uint32_t x = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += t;
            }
            if (lane == 31) wsum[warp] = x;
            __syncthreads();
            uint32_t before = 0;
            for (int w = 0; w < warp; w++) before += wsum[w];
            lstart[d] = before + x - cnt;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kItems; r++) {
            if (dig[r] >= 0) {
                const uint32_t lp = lstart[dig[r]] + wcnt[warp][dig[r]] + pos[r];
                sk[lp] = k[r];
                sv[lp] = v[r];
            }
        }
        // look back: keys of digit d in all earlier tiles.  The tiles of a
        // pass start together, so a walk that read one predecessor per L2
        // round trip would take about sqrt(2 tile) trips; each step reads a
        // window of kLook predecessors at once and sums them from the nearest
        // down to the first prefix, or up to the first tile that has not
        // published yet (read again next step).
        uint32_t excl = 0;
        if (tile > 0) {
            const volatile uint32_t* col = mine + d;
            int j = tile - 1;   // nearest tile not yet counted
            unsigned long long t0 = 0;
            for (;;) {
                uint32_t w[kLook];
#pragma unroll
                for (int q = 0; q < kLook; q++) w[q] = j - q >= 0 ? col[(size_t)(j - q) * kBins] : kFlagPre;
                int used = 0;
                bool done = false;
#pragma unroll
                for (int q = 0; q < kLook; q++) {
                    if (!done && used == q && (w[q] & (kFlagAgg | kFlagPre))) {
                        excl += w[q] & kCountMask;
                        used++;
                        done = (w[q] & kFlagPre) != 0;
                    }
                }
                if (done) break;
                j -= used;
                if (used == kLook) continue;
                // tile j has not published yet
                if (t0 == 0) {
                    t0 = sort_ns();
                } else if ((*(volatile int*)err & kErrSortStall) || sort_ns() - t0 > kLookLimitNs) {
                    atomicOr(err, kErrSortStall);
                    break;
                }
                __nanosleep(32);
            }
            row[d] = kFlagPre | ((excl + cnt) & kCountMask);
        }
        gstart[d] = digit_base + excl;
        __syncthreads();
        for (int j = threadIdx.x; j < tn; j += kThreads) {
            const uint64_t kk = sk[j];
            const uint32_t vv = sv[j];
            const int dd = kBoxDigit ? (int)((box[vv] >> shift) & 255) : (int)((kk >> shift) & 255ull);
            const uint32_t p = gstart[dd] + ((uint32_t)j - lstart[dd]);
            if (p < (uint32_t)n) {   // always true unless a look-back gave up
                kout[p] = kk;
                vout[p] = vv;
            }
        }
    }
}

// ---- int32 exclusive scan (3 phases) ----
constexpr int kScanTile = 2048;   // 256 threads x 8

__global__ void __launch_bounds__(256) k_scan_reduce(const int32_t* __restrict__ a, int ncap,
                                                     const int* d_n, int32_t* __restrict__ part) {
    const int n = d_n ? min(*d_n, ncap) : ncap;
    const int base = blockIdx.x * kScanTile;
    int s = 0;
#pragma unroll
    for (int r = 0; r < 8; r++) {
        int i = base + r * 256 + threadIdx.x;
        if (i < n) s += a[i];
    }
    __shared__ int ws[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < 8; w++) t += ws[w];
        part[blockIdx.x] = t;
    }
}

// Block scan of a 2048-element tile plus the tile's offset; a[n] = total.
__global__ void __launch_bounds__(256) k_scan_down(int32_t* __restrict__ a, int ncap,
                                                   const int* d_n,
                                                   const int32_t* __restrict__ part,
                                                   const int32_t* __restrict__ total) {
    const int n = d_n ? min(*d_n, ncap) : ncap;
    const int base = blockIdx.x * kScanTile;
    if (base > n) return;
    const int t0 = base + threadIdx.x * 8;
    int v[8];
    int s = 0;
#pragma unroll
    for (int r = 0; r < 8; r++) {
        int i = t0 + r;
        v[r] = i < n ? a[i] : 0;
        s += v[r];
    }
    __shared__ int ws[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    int wo = 0;
    for (int q = 0; q < w; q++) wo += ws[q];
    int run = part[blockIdx.x] + wo + x - s;
#pragma unroll
    for (int r = 0; r < 8; r++) {
        int i = t0 + r;
        if (i < n) a[i] = run;
        if (i == n) a[i] = *total;
        run += v[r];
    }
}

}  // namespace

// Digit totals of every pass, then two banks of per-tile status words.
size_t radix_hist_words(int ncap) {
    return (size_t)kMaxPasses * kBins +
           2 * (size_t)kBins * (size_t)ceil_div(ncap > 0 ? ncap : 1, kTile);
}

size_t scan_part_words(int ncap) { return (size_t)ceil_div((long long)ncap + 1, kScanTile) + 1; }

int radix_sort_passes(int key_bits, bool box_pass, int box_bits) {
    return ceil_div(key_bits, 8) + (box_pass ? ceil_div(box_bits, 8) : 0);
}

int radix_sort(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, int ncap, const int* d_n,
               int key_bits, const int32_t* box_digits, int box_bits, uint32_t* hist, int* err,
               cudaStream_t s) {
    if (ncap <= 0) return 0;
    const int tiles_cap = ceil_div(ncap, kTile);
    uint32_t* status = hist + kMaxPasses * kBins;
    const int passes_key = ceil_div(key_bits, 8);
    const int passes_box = box_digits ? ceil_div(box_bits, 8) : 0;
    // digit totals start at zero; the status banks are cleared by the
    // kernels, for the tiles in use only
    cudaMemsetAsync(hist, 0, sizeof(uint32_t) * kMaxPasses * kBins, s);
    const int hgrid = std::max(1, std::min(ceil_div(ncap, 8 * kThreads), 1024));
    if (box_digits)
        k_rs_hist<true><<<hgrid, kThreads, 0, s>>>(k0, v0, box_digits, d_n, ncap, passes_key,
                                                   passes_box, hist, status, tiles_cap);
    else
        k_rs_hist<false><<<hgrid, kThreads, 0, s>>>(k0, v0, nullptr, d_n, ncap, passes_key, 0, hist,
                                                    status, tiles_cap);
    int cur = 0;
    uint64_t* K[2] = {k0, k1};
    uint32_t* V[2] = {v0, v1};
    for (int p = 0; p < passes_key + passes_box; p++) {
        const bool boxp = p >= passes_key;
        const int sh = boxp ? 8 * (p - passes_key) : 8 * p;
        if (boxp)
            k_rs_pass<true><<<tiles_cap, kThreads, 0, s>>>(K[cur], V[cur], K[cur ^ 1], V[cur ^ 1],
                                                           box_digits, d_n, ncap, sh, p, hist,
                                                           status, tiles_cap, err);
        else
            k_rs_pass<false><<<tiles_cap, kThreads, 0, s>>>(K[cur], V[cur], K[cur ^ 1], V[cur ^ 1],
                                                            nullptr, d_n, ncap, sh, p, hist, status,
                                                            tiles_cap, err);
        cur ^= 1;
    }
    return cur;
}

void exclusive_scan_i32(int32_t* data, int n_cap, const int* d_n, int32_t* part, int32_t* total,
                        cudaStream_t s) {
    const int nb = ceil_div((long long)n_cap + 1, kScanTile);
    k_scan_reduce<<<nb, 256, 0, s>>>(data, n_cap, d_n, part);
    k_scan_block<int32_t><<<1, kScanThreads, 0, s>>>(part, nb, total);
    k_scan_down<<<nb, 256, 0, s>>>(data, n_cap, d_n, part, total);
}

}  // namespace rb
