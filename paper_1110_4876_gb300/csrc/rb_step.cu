// rb_step.cu -- the per-particle parts of a DKD step (Sect. 3): drift with
// boundaries (Sect. 2.3) fused with the Morton keys of the next tree build,
// the kick, the gather into Morton order, collision resolution (Sect. 5,
// Eq. 2) and the energy/momentum sums (Sect. 6.2).
//
// Drift, kick, boundary wrap, the overlap geometry and the resolution use
// explicitly rounded FP64 operations (__dadd_rn, __dmul_rn, ...) so the
// compiler never fuses them: they give bit-identical results to any other
// IEEE FP64 implementation that evaluates the same expressions in the same
// order without fused multiply-adds.
#include <algorithm>
#include <climits>

#include <cooperative_groups.h>

#include "rb_internal.cuh"

namespace cg = cooperative_groups;

namespace rb {
namespace {

__device__ __forceinline__ uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// Integer coordinate floor(((x - lo) / L) * 2^21), clamped to [0, 2^21 - 1].
// k = (x - lo) * scale, with scale = (1/L, rounded) x 2^21 (a power-of-two
// scaling, so no further rounding), lies within 2^-30 of the oracle's
// fl((x - lo) / L) x 2^21; wherever k is at least 2^-23 from every grid line
// both have the same floor.  For k in [1, 2^21) the floor and that distance
// are read from k's bits with integer operations: on GB300 an FP64
// instruction holds the SM's FP64 pipe 16 cycles per warp, and this kernel's
// time is its FP64 instructions.  Other k and the few near a grid line take
// the FP64 division.
__device__ __forceinline__ uint32_t icoord(double x, double lo, double L, double scale) {
    const double d = __dsub_rn(x, lo);
    const uint64_t b = (uint64_t)__double_as_longlong(__dmul_rn(d, scale));
    const int e = (int)(b >> 52) - 1023;   // unbiased exponent (sign set or NaN: e > 20)
    if (e >= 0 && e <= 20) {
        const int sh = 52 - e;             // fraction bits of k
        const uint64_t m = (b & 0xfffffffffffffull) | (1ull << 52);
        const uint64_t one = 1ull << sh, fr = m & (one - 1), tol = 1ull << (sh - 23);
        if (fr >= tol && one - fr >= tol) return (uint32_t)(m >> sh);
    }
    double k = floor(__dmul_rn(__ddiv_rn(d, L), 2097152.0));
    if (!(k >= 0.0)) k = 0.0;
    if (k > 2097151.0) k = 2097151.0;
    return (uint32_t)k;
}

// Order-preserving integer image of a double: for a, b not NaN (and -0 not
// compared with +0), a < b exactly when dord(a) < dord(b), and for h > 0,
// dord(-h) = ~dord(h).  The boundary tests compare this way, without FP64
// instructions.  A NaN coordinate compares as beyond every bound; the
// non-finite check after the wrap reports it either way.
__device__ __forceinline__ int64_t dord(double v) {
    const int64_t b = __double_as_longlong(v);
    return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}

__device__ __forceinline__ bool finite_bits(double v) {
    return ((__double_as_longlong(v) >> 52) & 0x7ff) != 0x7ff;
}

__device__ __forceinline__ double time_at(const Ctl* ctl, const SimC& C, int hs) {
    const double h = (double)(2 * ctl->step + hs);
    return __dadd_rn(C.t0, __dmul_rn(h, C.half_dt));
}

__device__ __forceinline__ void drift_one(const SimC& C, double& x, double& y, double& z,
                                          double& vx, double& vy, double& vz) {
    if (C.integrator == 0) {
        x = __dadd_rn(x, __dmul_rn(vx, C.half_dt));
        y = __dadd_rn(y, __dmul_rn(vy, C.half_dt));
        z = __dadd_rn(z, __dmul_rn(vz, C.half_dt));
        return;
    }
    const double x0 = x, u0 = vx, v0 = vy, z0 = z, w0 = vz;
    x = __dadd_rn(__dadd_rn(__dmul_rn(C.axx, x0), __dmul_rn(C.axu, u0)), __dmul_rn(C.axv, v0));
    y = __dadd_rn(y, __dadd_rn(__dadd_rn(__dmul_rn(C.ayx, x0), __dmul_rn(C.ayu, u0)),
                               __dmul_rn(C.ayv, v0)));
    vx = __dadd_rn(__dadd_rn(__dmul_rn(C.aux, x0), __dmul_rn(C.auu, u0)), __dmul_rn(C.auv, v0));
    vy = __dadd_rn(__dadd_rn(__dmul_rn(C.avx, x0), __dmul_rn(C.avu, u0)), __dmul_rn(C.avv, v0));
    z = __dadd_rn(__dmul_rn(C.azz, z0), __dmul_rn(C.azw, w0));
    vz = __dadd_rn(__dmul_rn(C.awz, z0), __dmul_rn(C.aww, w0));
}

// Wraps in y (and z) repeat the oracle's one-box-length steps; a particle
// that would need more than this many is reported as a runaway.
constexpr int kMaxWraps = 1 << 12;

// Boundaries after a drift half; returns false if the particle left an open
// boundary.  *runaway is set when the wraps did not bring it back.
__device__ __forceinline__ bool wrap_one(const SimC& C, const BoxP& bp, const Ctl* ctl, int hs, double& x,
                                         double& y, double& z, double& vy, bool* runaway) {
    const int64_t ux = dord(bp.hx), uy = dord(bp.hy), uz = dord(bp.hz);   // ~u is -h
    if (C.boundary == 0) {
        const int64_t ox = dord(x), oy = dord(y), oz = dord(z);
        return !(ox < ~ux || ox >= ux || oy < ~uy || oy >= uy || oz < ~uz || oz >= uz);
    }
    const double vs = bp.shear_speed;
    const int64_t ox = dord(x);
    const bool up = ox >= ux, down = ox < ~ux;
    // the shear offset only for the few particles that cross in x
    const double s = (up || down) && (__double_as_longlong(vs) << 1) != 0
                         ? fmod(__dmul_rn(vs, time_at(ctl, C, hs)), bp.Ly)
                         : 0.0;
    if (up) {
        x = __dsub_rn(x, bp.Lx);
        y = __dadd_rn(y, s);
        vy = __dadd_rn(vy, vs);
    } else if (down) {
        x = __dadd_rn(x, bp.Lx);
        y = __dsub_rn(y, s);
        vy = __dsub_rn(vy, vs);
    }
    for (int k = 0; k < kMaxWraps && dord(y) >= uy; k++) y = __dsub_rn(y, bp.Ly);
    for (int k = 0; k < kMaxWraps && dord(y) < ~uy; k++) y = __dadd_rn(y, bp.Ly);
    const int64_t oy = dord(y);
    if (oy >= uy || oy < ~uy) *runaway = true;
    if (C.z_periodic) {
        for (int k = 0; k < kMaxWraps && dord(z) >= uz; k++) z = __dsub_rn(z, bp.Lz);
        for (int k = 0; k < kMaxWraps && dord(z) < ~uz; k++) z = __dadd_rn(z, bp.Lz);
        const int64_t oz = dord(z);
        if (oz >= uz || oz < ~uz) *runaway = true;
        return true;
    }
    const int64_t oz = dord(z);
    return !(oz < ~uz || oz >= uz);
}

struct DriftArgs {
    PSet P;
    uint64_t* key;
    uint32_t* idx;
    int32_t* sbox;
    Ctl* ctl;
    const BoxP* boxes;
    const double *ax, *ay, *az;
    int ncap, ndrift, hs;
    bool kick;
};

// Optional kick (v += a dt), one or two drift halves each followed by the
// boundaries, then the Morton key of the new position for the next sort.
__global__ void __launch_bounds__(256) k_drift_keys(DriftArgs A, SimC C) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.ncap) return;
    A.idx[i] = (uint32_t)i;
    bool live = A.P.box[i] < C.nbox;
    uint64_t key = kRemovedKey;
    if (live) {
        double x = A.P.x[i], y = A.P.y[i], z = A.P.z[i];
        double vx = A.P.vx[i], vy = A.P.vy[i], vz = A.P.vz[i];
        const BoxP bp = A.boxes[A.P.box[i]];
        if (A.kick) {
            vx = __dadd_rn(vx, __dmul_rn(A.ax[i], C.dt));
            vy = __dadd_rn(vy, __dmul_rn(A.ay[i], C.dt));
            vz = __dadd_rn(vz, __dmul_rn(A.az[i], C.dt));
        }
        bool runaway = false;
        for (int d = 0; d < A.ndrift && live; d++) {
            drift_one(C, x, y, z, vx, vy, vz);
            live = wrap_one(C, bp, A.ctl, A.hs + d, x, y, z, vy, &runaway);
        }
        if (runaway || !(finite_bits(x) && finite_bits(y) && finite_bits(z))) {
            atomicOr(&A.ctl->err, kErrNonFinite);
            live = false;
        }
        A.P.x[i] = x; A.P.y[i] = y; A.P.z[i] = z;
        A.P.vx[i] = vx; A.P.vy[i] = vy; A.P.vz[i] = vz;
        if (live) {
            const double lo = -bp.hx;   // the root cube's side L is Lx
            key = (spread3(icoord(x, lo, bp.L, bp.key_scale)) << 2) |
                  (spread3(icoord(y, lo, bp.L, bp.key_scale)) << 1) |
                  spread3(icoord(z, lo, bp.L, bp.key_scale));
        }
    }
    A.key[i] = key;
    A.sbox[i] = live ? A.P.box[i] : C.nbox;
    if (!live) A.P.box[i] = C.nbox;
    const unsigned b = __ballot_sync(0xffffffffu, live);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(&A.ctl->n_live_next, __popc(b));
}

__global__ void __launch_bounds__(256) k_permute(PSet S, PSet D, const uint32_t* __restrict__ idx,
                                                 int32_t* __restrict__ slot_of_id, const Ctl* ctl,
                                                 int ncap) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncap) return;
    const int j = (int)idx[i];
    D.x[i] = S.x[j]; D.y[i] = S.y[j]; D.z[i] = S.z[j];
    D.vx[i] = S.vx[j]; D.vy[i] = S.vy[j]; D.vz[i] = S.vz[j];
    D.m[i] = S.m[j]; D.r[i] = S.r[j];
    const int id = S.id[j];
    D.id[i] = id;
    D.box[i] = S.box[j];
    if (i < ctl->n_live_next) slot_of_id[id] = i;
}

__global__ void k_commit_live(Ctl* ctl) {
    ctl->n_live = ctl->n_live_next;
    ctl->n_live_next = 0;
}

__global__ void k_discard_live(Ctl* ctl) { ctl->n_live_next = 0; }

// An overflowing search resolves nothing: the host grows the buffer and runs
// the search again on the unchanged state.
__global__ void k_pairs_prep(Ctl* ctl, int cap) {
    const int c = ctl->pair_count;
    const int n = c <= cap ? c : 0;
    ctl->pair_n = n;
    ctl->pair_ends = 2 * n;
    ctl->pending = n;
    ctl->resolved = 0;
}

struct ResolveArgs {
    PSet P;
    const uint64_t* key;
    const int32_t* slot_of_id;
    const int32_t *prev_a, *prev_b;   // previous pair of particle a / b (queue order), or -1
    const int32_t *next_a, *next_b;   // next pair of particle a / b, or -1
    int32_t* wait;                    // predecessors of a pair not yet resolved
    Ctl* ctl;
    const BoxP* boxes;
    int hs;
    const ImgTab* img;   // [box][image] offsets at the detection time
    int nimg, ngx, ngy, ngz;
};

__device__ __forceinline__ void pair_slots(const ResolveArgs& A, uint64_t k, int& sa, int& sb) {
    sa = A.slot_of_id[(int)(k >> 36)];
    sb = A.slot_of_id[(int)((k >> 12) & 0xFFFFFFull)];
}

// Eq. 2 for one pair, in the oracle's operation order.  kCG: velocities are
// read from L2 (other SMs update them while the queue runs).
template <bool kCG = false>
__device__ __forceinline__ bool resolve_one(const ResolveArgs& A, const SimC& C, uint64_t k) {
    int a, b;
    pair_slots(A, k, a, b);
    const int code = (int)(k & 0xFFFull);
    const int gx = (code & 15) - 7, gy = ((code >> 4) & 15) - 7, gz = ((code >> 8) & 15) - 7;
    // the image's offsets from the table (same formulas as the search used)
    const int g = ((gx + A.ngx) * (2 * A.ngy + 1) + (gy + A.ngy)) * (2 * A.ngz + 1) + (gz + A.ngz);
    const ImgTab& T = A.img[(size_t)A.P.box[a] * A.nimg + g];
    const double ox = T.ox, oy = T.oy, oz = T.oz, dvg = T.dvy;
    const double rx = __dsub_rn(__dadd_rn(A.P.x[b], ox), A.P.x[a]);
    const double ry = __dsub_rn(__dadd_rn(A.P.y[b], oy), A.P.y[a]);
    const double rz = __dsub_rn(__dadd_rn(A.P.z[b], oz), A.P.z[a]);
    double vxa, vya, vza, vxb, vyb, vzb;
    if (kCG) {
        vxa = __ldcg(&A.P.vx[a]); vya = __ldcg(&A.P.vy[a]); vza = __ldcg(&A.P.vz[a]);
        vxb = __ldcg(&A.P.vx[b]); vyb = __ldcg(&A.P.vy[b]); vzb = __ldcg(&A.P.vz[b]);
    } else {
        vxa = A.P.vx[a]; vya = A.P.vy[a]; vza = A.P.vz[a];
        vxb = A.P.vx[b]; vyb = A.P.vy[b]; vzb = A.P.vz[b];
    }
    const double ux = __dsub_rn(vxb, vxa), uy = __dsub_rn(__dadd_rn(vyb, dvg), vya),
                 uz = __dsub_rn(vzb, vza);
    const double rv = __dadd_rn(__dadd_rn(__dmul_rn(rx, ux), __dmul_rn(ry, uy)), __dmul_rn(rz, uz));
    if (rv >= 0.0) return false;
    // the impulse along n = r/|r| without forming n: v_a gains
    // (1 + eps) (m_b/M) (u.r)/|r|^2 r, v_b loses the same with m_a (one
    // division, no square root: GB300's FP64 rate is 1/64 of FP32)
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(rx, rx), __dmul_rn(ry, ry)), __dmul_rn(rz, rz));
    double e = C.eps;
    if (C.eps_law == 1) {
        // velocity-dependent restitution: min(1, (|v_n| / v_c)^(-p)), |v_n| = |u.r| / |r|
        const double vn = __ddiv_rn(rv, __dsqrt_rn(r2));
        const double q = pow(__ddiv_rn(fabs(vn), C.eps_vc), -C.eps_p);
        e = q < 1.0 ? q : 1.0;
    }
    const double ma = A.P.m[a], mb = A.P.m[b];
    const double mt = __dadd_rn(ma, mb);
    const double gi = __ddiv_rn(__dmul_rn(__dadd_rn(1.0, e), rv), __dmul_rn(r2, mt));
    const double ga = __dmul_rn(gi, mb), gb = __dmul_rn(gi, ma);
    A.P.vx[a] = __dadd_rn(vxa, __dmul_rn(ga, rx));
    A.P.vy[a] = __dadd_rn(vya, __dmul_rn(ga, ry));
    A.P.vz[a] = __dadd_rn(vza, __dmul_rn(ga, rz));
    A.P.vx[b] = __dsub_rn(vxb, __dmul_rn(gb, rx));
    A.P.vy[b] = __dsub_rn(vyb, __dmul_rn(gb, ry));
    A.P.vz[b] = __dsub_rn(vzb, __dmul_rn(gb, rz));
    return true;
}

// Pair ends for the predecessor links: (particle slot, 2 * pair + side).
__global__ void __launch_bounds__(256) k_pair_ends(ResolveArgs A, uint64_t* __restrict__ ekey,
                                                   uint32_t* __restrict__ eval) {
    const int n = A.ctl->pair_n;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        int a, b;
        pair_slots(A, A.key[k], a, b);
        ekey[2 * k] = (uint64_t)a;
        ekey[2 * k + 1] = (uint64_t)b;
        eval[2 * k] = 2u * k;
        eval[2 * k + 1] = 2u * k + 1u;
    }
}

// After a stable sort of the ends by particle, consecutive ends of the same
// particle are consecutive pairs of that particle in queue order.
__global__ void __launch_bounds__(256) k_pair_prev(const uint64_t* __restrict__ ekey,
                                                   const uint32_t* __restrict__ eval,
                                                   const Ctl* __restrict__ ctl,
                                                   int32_t* __restrict__ prev_a,
                                                   int32_t* __restrict__ prev_b,
                                                   int32_t* __restrict__ next_a,
                                                   int32_t* __restrict__ next_b) {
    const int m = ctl->pair_ends;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x) {
        const uint32_t v = eval[e];
        const int k = (int)(v >> 1);
        const int prev = (e > 0 && ekey[e - 1] == ekey[e]) ? (int)(eval[e - 1] >> 1) : -1;
        const int next = (e + 1 < m && ekey[e + 1] == ekey[e]) ? (int)(eval[e + 1] >> 1) : -1;
        if (v & 1u) {
            prev_b[k] = prev;
            next_b[k] = next;
        } else {
            prev_a[k] = prev;
            next_a[k] = next;
        }
    }
}

// The queue's first slots: the pairs that are the first pair of both their
// particles; every pair waits for as many predecessors as it has.
// One atomic per block and pass: the block's ready pairs are ranked with a
// block scan of warp ballots (their order in the queue does not matter).
__global__ void __launch_bounds__(256) k_res_seed(ResolveArgs A, SimC C, int32_t* __restrict__ list,
                                                  int32_t* __restrict__ rcnt) {
    __shared__ int wcount[8], base;
    const int n = A.ctl->pair_n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k0 = blockIdx.x * blockDim.x; k0 < n; k0 += gridDim.x * blockDim.x) {
        const int k = k0 + threadIdx.x;
        bool ready = false;
        if (k < n) {
            const int w = (A.prev_a[k] >= 0 ? 1 : 0) + (A.prev_b[k] >= 0 ? 1 : 0) +
                          (C.hold_pair && k == 0 ? 1 : 0);
            A.wait[k] = w;
            ready = w == 0;
        }
        const unsigned m = __ballot_sync(0xffffffffu, ready);
        if (lane == 0) wcount[warp] = __popc(m);
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int q = 0; q < (int)(blockDim.x >> 5); q++) t += wcount[q];
            base = t ? atomicAdd(&rcnt[0], t) : 0;
        }
        __syncthreads();
        if (ready) {
            int pos = base + __popc(m & ((1u << lane) - 1u));
            for (int q = 0; q < warp; q++) pos += wcount[q];
            list[pos] = k;
        }
        __syncthreads();   // wcount and base are reused
    }
}

// The queue of ready pairs, worked by every resident thread in one launch.
// A pair enters the queue (after the seed's pairs, in the order they become
// ready) once every earlier pair of the sorted queue that shares a particle
// with it is resolved; its wait count of unresolved predecessors reaches zero
// at the release of the last one.  Threads claim queue slots in order (32
// per warp vote) and wait for their slot to be written; a slot is written by
// the thread that released its pair, after the velocities it wrote are made
// visible (fence), and the velocities are read from L2.  Every pair sees all
// earlier pairs that share a particle with it, so the outcome equals
// resolving the sorted queue one pair at a time.  The claims are in queue
// order and a thread resolves its pair as soon as the slot is written, so
// the wait ends however many of the launch's blocks are resident (slots are
// claimed only by running threads); it is bounded all the same (half a
// second), and reports kErrResolveStall if it ever gives up.
constexpr unsigned long long kWaitLimitNs = 500000000ull;   // half a second

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void queue_push(int32_t* list, int32_t* tail, int k) {
    cg::coalesced_group g = cg::coalesced_threads();
    int base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(tail, (int)g.size());
    *(volatile int32_t*)&list[g.shfl(base, 0) + (int)g.thread_rank()] = k;
}

__global__ void __launch_bounds__(256) k_res_queue(ResolveArgs A, SimC C, int32_t* __restrict__ list,
                                                   int32_t* __restrict__ q) {
    // q[0]: slots written (the seed's pairs first), q[1]: slots claimed
    const int np = A.ctl->pair_n;
    const int lane = threadIdx.x & 31;
    int nres = 0, ndone = 0;
    for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(&q[1], 32);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= np) break;
        const int idx = base + lane;
        bool stalled = false;
        if (idx < np) {
            int k = *(volatile int32_t*)&list[idx];
            const unsigned long long t0 = k < 0 ? global_ns() : 0ull;
            while (k < 0) {
                // bounded: half a second, or at once when another thread gave up
                if ((*(volatile int*)&A.ctl->err & kErrResolveStall) || global_ns() - t0 > kWaitLimitNs) {
                    atomicOr(&A.ctl->err, kErrResolveStall);
                    stalled = true;
                    break;
                }
                __nanosleep(200);
                k = *(volatile int32_t*)&list[idx];
            }
            if (!stalled) {
                __threadfence();   // the releasing thread's velocities before ours
                nres += resolve_one<true>(A, C, A.key[k]) ? 1 : 0;
                ndone++;
                __threadfence();   // our velocities before the successors are released
                const int na = A.next_a[k], nb = A.next_b[k];
                if (na >= 0 && atomicSub(&A.wait[na], 1) == 1) queue_push(list, &q[0], na);
                if (nb >= 0 && atomicSub(&A.wait[nb], 1) == 1) queue_push(list, &q[0], nb);
            }
        }
        if (__any_sync(0xffffffffu, stalled)) break;
    }
    if (ndone) atomicSub(&A.ctl->pending, ndone);
    if (nres) atomicAdd(&A.ctl->resolved, nres);
}

int g_queue_blocks = 0;   // resident blocks of k_res_queue on the whole GPU

}  // namespace

void resolve_prepare(int nsm) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_res_queue, 256, 0) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
    }
    g_queue_blocks = std::max(nsm, 1) * std::max(per_sm, 1);
}

namespace {

__global__ void k_step_advance(Ctl* ctl) { ctl->step += 1; }

// Energy terms of one box, per block: K, tidal, W, Px, Py, Pz, count.
__global__ void __launch_bounds__(256) k_energy_partial(PSet P, const Ctl* ctl, SimC C,
                                                        const double* __restrict__ phi, int box,
                                                        double* __restrict__ partials) {
    const int n = ctl->n_live;
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (P.box[i] != box) continue;
        const double m = P.m[i];
        const double vx = P.vx[i], vy = P.vy[i], vz = P.vz[i];
        s[0] += 0.5 * m * (vx * vx + vy * vy + vz * vz);
        if (C.integrator == 1)
            s[1] += m * (0.5 * (C.omega_z * C.omega_z) * (P.z[i] * P.z[i]) -
                          1.5 * (C.omega * C.omega) * (P.x[i] * P.x[i]));
        if (phi) s[2] += 0.5 * m * phi[i];
        s[3] += m * vx;
        s[4] += m * vy;
        s[5] += m * vz;
        s[6] += 1.0;
    }
    __shared__ double red[7][8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 7; q++) {
        double v = s[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[q][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        double v = 0.0;
        for (int k = 0; k < 8; k++) v += red[threadIdx.x][k];
        partials[threadIdx.x * gridDim.x + blockIdx.x] = v;
    }
}

__global__ void k_energy_final(const double* __restrict__ partials, int nparts,
                               double* __restrict__ out7) {
    const int q = threadIdx.x;
    if (q >= 7) return;
    double v = 0.0;
    for (int k = 0; k < nparts; k++) v += partials[q * nparts + k];
    out7[q] = v;
}

}  // namespace

void drift_keys(const PSet& P, const Tree& T, Ctl* ctl, const BoxP* boxes, const SimC& C,
                int ncap, int ndrift, int half_step_offset, const double* ax, const double* ay,
                const double* az, bool kick, cudaStream_t s) {
    if (ncap <= 0) return;
    DriftArgs A;
    A.P = P; A.key = T.key; A.idx = T.idx; A.sbox = T.sbox; A.ctl = ctl; A.boxes = boxes;
    A.ax = ax; A.ay = ay; A.az = az;
    A.ncap = ncap; A.ndrift = ndrift; A.hs = half_step_offset; A.kick = kick;
    k_drift_keys<<<ceil_div(ncap, 256), 256, 0, s>>>(A, C);
}

void sort_and_permute(const PSet& src, const PSet& dst, Tree& T, Pairs& PR, Ctl* ctl,
                      const SimC& C, int ncap, int box_bits, cudaStream_t s) {
    if (ncap <= 0) return;
    const int which = radix_sort(T.key, T.idx, T.key_alt, T.idx_alt, ncap, nullptr, 64,
                                 C.nbox > 1 ? T.sbox : nullptr, box_bits, T.hist, &ctl->err, s);
    if (which == 1) {
        // keep the sorted keys in T.key for the topology kernels
        uint64_t* k = T.key; T.key = T.key_alt; T.key_alt = k;
        uint32_t* v = T.idx; T.idx = T.idx_alt; T.idx_alt = v;
    }
    k_permute<<<ceil_div(ncap, 256), 256, 0, s>>>(src, dst, T.idx, PR.slot_of_id, ctl, ncap);
    k_commit_live<<<1, 1, 0, s>>>(ctl);
}

void discard_live_count(Ctl* ctl, cudaStream_t s) { k_discard_live<<<1, 1, 0, s>>>(ctl); }

// Live particles of one box written in id order (id - base) to out, with a
// flag per id and a count.
__global__ void __launch_bounds__(256) k_by_id(PSet P, PSet out, int box, int base, int ncap,
                                               int32_t* __restrict__ flags, int* __restrict__ count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool mine = i < ncap && P.box[i] == box;
    if (mine) {
        const int k = P.id[i] - base;
        out.x[k] = P.x[i]; out.y[k] = P.y[i]; out.z[k] = P.z[i];
        out.vx[k] = P.vx[i]; out.vy[k] = P.vy[i]; out.vz[k] = P.vz[i];
        out.m[k] = P.m[i]; out.r[k] = P.r[i];
        flags[k] = 1;
    }
    const unsigned b = __ballot_sync(0xffffffffu, mine);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(count, __popc(b));
}

// Slots of a freshly copied single box: slot i holds id i; slots from n on
// are unused (box = nbox).
__global__ void __launch_bounds__(256) k_reset_slots(PSet P, int32_t* __restrict__ slot_of_id, int n,
                                                     int ncap, int nbox) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncap) return;
    P.id[i] = i;
    P.box[i] = i < n ? 0 : nbox;
    slot_of_id[i] = i;
}

// Checks of freshly copied particles: bit 0 a non-finite position or
// velocity, bit 1 a negative (or NaN) mass or radius; the largest radius as
// the bits of a non-negative double.
__global__ void __launch_bounds__(256) k_check_particles(PSet P, int n,
                                                         unsigned long long* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long bad = 0, rb = 0;
    if (i < n) {
        if (!(isfinite(P.x[i]) && isfinite(P.y[i]) && isfinite(P.z[i]) && isfinite(P.vx[i]) &&
              isfinite(P.vy[i]) && isfinite(P.vz[i])))
            bad |= 1ull;
        const double r = P.r[i];
        if (!(P.m[i] >= 0.0) || !(r >= 0.0)) bad |= 2ull;
        else if (r > 0.0) rb = (unsigned long long)__double_as_longlong(r);   // not -0.0
    }
    for (int o = 16; o > 0; o >>= 1) {
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
        rb = max(rb, __shfl_xor_sync(0xffffffffu, rb, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (bad) atomicOr(&out[0], bad);
        if (rb) atomicMax(&out[1], rb);
    }
}

void check_particles(const PSet& P, int n, unsigned long long* out2, cudaStream_t s) {
    cudaMemsetAsync(out2, 0, 2 * sizeof(unsigned long long), s);
    if (n > 0) k_check_particles<<<ceil_div(n, 256), 256, 0, s>>>(P, n, out2);
}

void particles_by_id(const PSet& P, const PSet& out, int box, int base, int ncap, int32_t* flags,
                     int nflags, int* count, cudaStream_t s) {
    cudaMemsetAsync(flags, 0, sizeof(int32_t) * (size_t)(nflags > 0 ? nflags : 1), s);
    cudaMemsetAsync(count, 0, sizeof(int), s);
    if (ncap > 0) k_by_id<<<ceil_div(ncap, 256), 256, 0, s>>>(P, out, box, base, ncap, flags, count);
}

void reset_slots(const PSet& P, int32_t* slot_of_id, int n, int ncap, int nbox, cudaStream_t s) {
    if (ncap > 0) k_reset_slots<<<ceil_div(ncap, 256), 256, 0, s>>>(P, slot_of_id, n, ncap, nbox);
}

void sort_pairs(Pairs& PR, Ctl* ctl, cudaStream_t s, int key_bits) {
    k_pairs_prep<<<1, 1, 0, s>>>(ctl, PR.cap);
    // an odd number of passes leaves the keys in key_alt; the buffers are
    // not swapped, so every captured graph finds them in the same place
    PR.sorted_alt = radix_sort(PR.key, PR.val, PR.key_alt, PR.val_alt, PR.cap, &ctl->pair_n,
                               key_bits, nullptr, 0, PR.hist, &ctl->err, s) == 1;
}

void resolve_pairs(const PSet& P, Ctl* ctl, const BoxP* boxes, const SimC& C, Pairs& PR,
                   int half_step_offset, ImgTab* img, cudaStream_t s) {
    ResolveArgs A;
    A.P = P; A.key = PR.sorted(); A.slot_of_id = PR.slot_of_id;
    A.prev_a = PR.prev_a; A.prev_b = PR.prev_b;
    A.next_a = PR.next_a; A.next_b = PR.next_b; A.wait = PR.wait;
    A.img = img;
    A.ngx = C.ngx; A.ngy = C.ngy; A.ngz = C.ngz;
    A.nimg = build_image_table(boxes, ctl, C, half_step_offset, img, s);
    A.ctl = ctl; A.boxes = boxes; A.hs = half_step_offset;
    const int grid = std::min(ceil_div(PR.cap, 256), 4 * 152);
    k_pair_ends<<<grid, 256, 0, s>>>(A, PR.ekey, PR.eval);
    // particle slots are < 2^24: three 8-bit passes, stable in queue order
    const int which = radix_sort(PR.ekey, PR.eval, PR.ekey_alt, PR.eval_alt, 2 * PR.cap,
                                 &ctl->pair_ends, 24, nullptr, 0, PR.ehist, &ctl->err, s);
    k_pair_prev<<<2 * grid, 256, 0, s>>>(which ? PR.ekey_alt : PR.ekey,
                                         which ? PR.eval_alt : PR.eval, ctl, PR.prev_a, PR.prev_b,
                                         PR.next_a, PR.next_b);
    cudaMemsetAsync(PR.rcnt, 0, sizeof(int32_t) * 64, s);
    cudaMemsetAsync(PR.queue, 0xff, sizeof(int32_t) * (size_t)PR.cap, s);   // every slot unwritten
    k_res_seed<<<grid, 256, 0, s>>>(A, C, PR.queue, PR.rcnt);
    // resident blocks only: a thread may wait for a slot that another writes
    const int qgrid = std::max(1, std::min(ceil_div(PR.cap, 256), g_queue_blocks));
    k_res_queue<<<qgrid, 256, 0, s>>>(A, C, PR.queue, PR.rcnt);
}

void energy_terms(const PSet& P, Ctl* ctl, const SimC& C, const double* phi, int box,
                  double* partials, int nparts, double* out7, cudaStream_t s) {
    k_energy_partial<<<nparts, 256, 0, s>>>(P, ctl, C, phi, box, partials);
    k_energy_final<<<1, 32, 0, s>>>(partials, nparts, out7);
}

void step_advance(Ctl* ctl, cudaStream_t s) { k_step_advance<<<1, 1, 0, s>>>(ctl); }

// The walk's counters (n_cell .. n_iter) and the search's (n_visit, n_siter).
void clear_walk_stats(Ctl* ctl, cudaStream_t s) {
    cudaMemsetAsync(&ctl->n_cell, 0, 7 * sizeof(unsigned long long), s);
}

void clear_search_stats(Ctl* ctl, cudaStream_t s) {
    cudaMemsetAsync(&ctl->n_visit, 0, 2 * sizeof(unsigned long long), s);
}

}  // namespace rb
