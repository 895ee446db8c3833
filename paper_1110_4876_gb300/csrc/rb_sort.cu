// rb_sort.cu -- stable LSD radix sort of (64-bit key, 32-bit value) pairs and
// an exclusive scan of int32 arrays, both sized on the device.
//
// The sort replaces the insertion/reconstruction of the paper's tree
// (Sect. 4.2): particles are put in Morton order so that every cell is a
// contiguous range.  Each 8-bit digit pass is three launches: per-tile digit
// counts (upsweep), one scan of the counts in digit-major order, and a
// stable scatter (downsweep) that ranks keys within a tile with warp
// match-any votes.  No pass waits on another block, so nothing can spin.
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

template <bool kBoxDigit>
__global__ void __launch_bounds__(kThreads) k_rs_up(const uint64_t* __restrict__ key,
                                                    const uint32_t* __restrict__ val,
                                                    const int32_t* __restrict__ box, const int* d_n,
                                                    int ncap, int shift, uint32_t* __restrict__ hist,
                                                    int nblocks) {
    __shared__ uint32_t h[kBins];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int n = read_n(d_n, ncap);
    const int base = blockIdx.x * kTile;
    const unsigned lt = (1u << (threadIdx.x & 31)) - 1u;
#pragma unroll 4
    for (int r = 0; r < kItems; r++) {
        const int i = base + r * kThreads + threadIdx.x;
        const bool ok = i < n;
        uint32_t d = 0;
        if (ok)
            d = kBoxDigit ? (uint32_t)(box[val[i]] >> shift) & 255u : (uint32_t)(key[i] >> shift) & 255u;
        // one shared atomic per distinct digit of the warp (nearly sorted
        // keys share their high digits)
        const unsigned act = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            const unsigned peers = __match_any_sync(act, d);
            if ((peers & lt) == 0) atomicAdd(&h[d], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    hist[threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// One block per digit: exclusive scan of that digit's per-tile counts (a
// contiguous row of the digit-major histogram) and the digit's total.
__global__ void __launch_bounds__(256) k_digit_rows(uint32_t* __restrict__ hist, int nblocks,
                                                    uint32_t* __restrict__ dtot) {
    __shared__ uint32_t wsum[8];
    uint32_t* row = hist + (size_t)blockIdx.x * nblocks;
    const int per = (nblocks + 255) / 256;
    const int b = threadIdx.x * per, e = min(b + per, nblocks);
    uint32_t s = 0;
    for (int i = b; i < e; i++) s += row[i];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t v = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) wsum[w] = v;
    __syncthreads();
    uint32_t run = v - s;
    for (int q = 0; q < w; q++) run += wsum[q];
    for (int i = b; i < e; i++) {
        const uint32_t c = row[i];
        row[i] = run;
        run += c;
    }
    if (threadIdx.x == 255) dtot[blockIdx.x] = run;
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

// Stable scatter of one tile: ranks within the tile (warp match-any votes),
// a local sort of the tile by digit in shared memory, then writes in local
// order, so that consecutive threads store consecutive addresses of a digit.
template <bool kBoxDigit>
__global__ void __launch_bounds__(kThreads) k_rs_down(const uint64_t* __restrict__ kin,
                                                      const uint32_t* __restrict__ vin,
                                                      uint64_t* __restrict__ kout,
                                                      uint32_t* __restrict__ vout,
                                                      const int32_t* __restrict__ box,
                                                      const int* d_n, int ncap, int shift,
                                                      const uint32_t* __restrict__ hist,
                                                      const uint32_t* __restrict__ dtot,
                                                      int nblocks) {
    __shared__ uint32_t wcnt[kThreads / 32][kBins];
    __shared__ uint32_t gstart[kBins];   // where digit d of this tile starts in the output
    __shared__ uint32_t lstart[kBins];   // where digit d starts inside the tile
    __shared__ uint32_t wsum[kThreads / 32];
    __shared__ uint64_t sk[kTile];
    __shared__ uint32_t sv[kTile];
    const int n = read_n(d_n, ncap);
    const int base = blockIdx.x * kTile;
    if (base >= n) return;
    const int tn = min(kTile, n - base);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = threadIdx.x; d < (kThreads / 32) * kBins; d += kThreads) (&wcnt[0][0])[d] = 0;
    {
        // start of digit d = (keys of all smaller digits) + (keys of digit d in
        // earlier tiles); the first is an exclusive scan of the digit totals
        const uint32_t tot = dtot[threadIdx.x];
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
        gstart[threadIdx.x] = before + v - tot + hist[threadIdx.x * nblocks + blockIdx.x];
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    uint64_t k[kItems];
    uint32_t v[kItems];
    uint32_t pos[kItems];
    int dig[kItems];
    const int wbase = base + warp * (kTile / (kThreads / 32));
#pragma unroll
    for (int r = 0; r < kItems; r++) {
        const int i = wbase + r * 32 + lane;
        const bool ok = i < n;
        k[r] = ok ? kin[i] : 0ull;
        v[r] = ok ? vin[i] : 0u;
        int d = 0;
        if (ok) d = kBoxDigit ? (int)((box[v[r]] >> shift) & 255) : (int)((k[r] >> shift) & 255ull);
        dig[r] = ok ? d : -1;
        const unsigned act = __ballot_sync(0xffffffffu, ok);
        pos[r] = 0;
        if (ok) {
            const unsigned peers = __match_any_sync(act, d);
            const int rank = __popc(peers & lt);
            const uint32_t c = wcnt[warp][d];
            pos[r] = c + rank;
            __syncwarp(act);
            if (rank == 0) wcnt[warp][d] = c + __popc(peers);
            __syncwarp(act);
        }
    }
    __syncthreads();
    {
        // digit d: offsets of each warp's keys inside the digit, the tile's
        // count, and the digit's start in the tile (block scan of the counts)
        const int d = threadIdx.x;
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; w++) {
            const uint32_t x = wcnt[w][d];
            wcnt[w][d] = c;
            c += x;
        }
        uint32_t x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        __syncthreads();   // wsum is reused
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        uint32_t before = 0;
        for (int w = 0; w < warp; w++) before += wsum[w];
        lstart[d] = before + x - c;
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
    __syncthreads();
    for (int j = threadIdx.x; j < tn; j += kThreads) {
        const uint64_t kk = sk[j];
        const uint32_t vv = sv[j];
        const int d = kBoxDigit ? (int)((box[vv] >> shift) & 255) : (int)((kk >> shift) & 255ull);
        const uint32_t p = gstart[d] + ((uint32_t)j - lstart[d]);
        kout[p] = kk;
        vout[p] = vv;
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

// Digit-major per-tile histogram plus 256 digit totals.
size_t radix_hist_words(int ncap) {
    return (size_t)kBins * (size_t)ceil_div(ncap > 0 ? ncap : 1, kTile) + kBins;
}

size_t scan_part_words(int ncap) { return (size_t)ceil_div((long long)ncap + 1, kScanTile) + 1; }

int radix_sort_passes(int key_bits, bool box_pass, int box_bits) {
    return ceil_div(key_bits, 8) + (box_pass ? ceil_div(box_bits, 8) : 0);
}

int radix_sort(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, int ncap, const int* d_n,
               int key_bits, const int32_t* box_digits, int box_bits, uint32_t* hist,
               cudaStream_t s) {
    if (ncap <= 0) return 0;
    const int nblocks = ceil_div(ncap, kTile);
    uint32_t* dtot = hist + (size_t)kBins * nblocks;
    int cur = 0;
    uint64_t* K[2] = {k0, k1};
    uint32_t* V[2] = {v0, v1};
    const int passes_key = ceil_div(key_bits, 8);
    const int passes_box = box_digits ? ceil_div(box_bits, 8) : 0;
    for (int p = 0; p < passes_key + passes_box; p++) {
        const bool boxp = p >= passes_key;
        const int sh = boxp ? 8 * (p - passes_key) : 8 * p;
        if (boxp)
            k_rs_up<true><<<nblocks, kThreads, 0, s>>>(K[cur], V[cur], box_digits, d_n, ncap, sh,
                                                       hist, nblocks);
        else
            k_rs_up<false><<<nblocks, kThreads, 0, s>>>(K[cur], V[cur], nullptr, d_n, ncap, sh,
                                                        hist, nblocks);
        k_digit_rows<<<kBins, 256, 0, s>>>(hist, nblocks, dtot);
        if (boxp)
            k_rs_down<true><<<nblocks, kThreads, 0, s>>>(K[cur], V[cur], K[cur ^ 1], V[cur ^ 1],
                                                         box_digits, d_n, ncap, sh, hist, dtot,
                                                         nblocks);
        else
            k_rs_down<false><<<nblocks, kThreads, 0, s>>>(K[cur], V[cur], K[cur ^ 1], V[cur ^ 1],
                                                          nullptr, d_n, ncap, sh, hist, dtot,
                                                          nblocks);
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
