// rb_sweep.cu -- plane-sweep collision detection along x (Sect. 5.3).
//
// The paper's sweep moves a plane through the 2N sorted x extents of the
// particle trajectories, keeps the list of trajectories the plane cuts, and
// tests each trajectory entering the list against every one already in it.
// On the GPU the same pair set comes from "sort and sweep":
//   1. every live particle gives an item: its trajectory's x extent
//      [x - |v_x| dt/2 - R - m, x + |v_x| dt/2 + R + m] (m = 1e-9 Lx), plus
//      copies shifted by +k Lx (k = 1..nghost_x) for ghost images across the
//      x boundary, emitted only when they can reach the box's own items;
//   2. items are radix-sorted by (box, quantised lower end);
//   3. one thread per sorted item P scans forward while the next item's lower
//      end is not beyond P's upper end: those are exactly the items whose
//      extents overlap P's and start after it, the trajectories already in the
//      paper's list when P enters it.  Each candidate (at least one original
//      particle, two different particles) is tested with the straight-line
//      criterion over every y/z image, in FP64 with the oracle's operation
//      sequence, on the canonical orientation (lower id a, image of b).
// The quantisation is a monotone map of the FP64 extents, so the scan never
// stops before an overlapping item; the exact FP64 comparison of the extents
// and a conservative y test only prune candidates the criterion rejects.
#include <cooperative_groups.h>

#include "rb_internal.cuh"

namespace cg = cooperative_groups;

namespace rb {
namespace {

constexpr double kMarginRel = 1e-9;   // extents widened by 1e-9 Lx (reading S3)

struct SweepArgs {
    PSet P;
    Ctl* ctl;
    const BoxP* boxes;
    uint64_t* key;
    uint32_t* val;
    uint64_t* pair_key;
    int pair_cap, item_cap, ncap, nbox;
    int ngx, ngy, ngz, hs;
    double t0, half_dt, h;   // h = dt / 2: the trajectory's half length in time
};

__device__ __forceinline__ double ext_of(const SweepArgs& A, int i) {
    return __dadd_rn(__dmul_rn(fabs(A.P.vx[i]), A.h), A.P.r[i]);
}

// Largest half extent |v_x| dt/2 + R over the live particles, as the bits of
// a non-negative double (ordered like the values).
__global__ void __launch_bounds__(256) k_sweep_ext(SweepArgs A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = min(A.ctl->n_live, A.ncap);
    unsigned long long b = 0ull;
    if (i < n && A.P.box[i] < A.nbox) b = (unsigned long long)__double_as_longlong(ext_of(A, i));
    for (int o = 16; o > 0; o >>= 1) b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
    if ((threadIdx.x & 31) == 0 && b) atomicMax(&A.ctl->sweep_wbits, b);
}

// Quantised position of v in a box's sweep range [base, base + span):
// floor((v - base) * 2^32 / span), clamped; monotone in v.
__device__ __forceinline__ uint64_t quant(double v, double base, double scale) {
    const double q = floor(__dmul_rn(__dsub_rn(v, base), scale));
    if (!(q > 0.0)) return 0ull;
    if (q >= 4294967295.0) return 4294967295ull;
    return (uint64_t)q;
}

struct Range {
    double base, scale, top, lx, m;
};

__device__ __forceinline__ Range range_of(const SweepArgs& A, const BoxP& bp) {
    Range g;
    const double w = __longlong_as_double((long long)A.ctl->sweep_wbits);
    g.lx = bp.Lx;
    g.m = kMarginRel * bp.Lx;
    const double W = w + g.m;
    g.base = -0.5 * bp.Lx - W;
    g.top = 0.5 * bp.Lx + W;
    g.scale = 4294967296.0 / (bp.Lx + 2.0 * W);
    return g;
}

// Items: the particle and its copies shifted by +k Lx that can reach the box.
// Each warp reserves its items with one atomic (prefix sum of the lanes'
// counts).
__global__ void __launch_bounds__(256) k_sweep_items(SweepArgs A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int n = min(A.ctl->n_live, A.ncap);
    int b = 0, cnt = 0;
    double lo0 = 0.0;
    Range g{};
    if (i < n) {
        b = A.P.box[i];
        if (b < A.nbox) {
            g = range_of(A, A.boxes[b]);
            lo0 = __dsub_rn(A.P.x[i], __dadd_rn(ext_of(A, i), g.m));
            cnt = 1;
            // copies k = 1..ngx whose lower end can still reach the box's items
            for (int k = 1; k <= A.ngx; k++) {
                if (__dadd_rn(lo0, __dmul_rn((double)k, g.lx)) > g.top) break;
                cnt++;
            }
        }
    }
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    int base = 0;
    if (lane == 31 && incl) base = atomicAdd(&A.ctl->sweep_items, incl);
    base = __shfl_sync(0xffffffffu, base, 31) + incl - cnt;
    for (int k = 0; k < cnt; k++) {
        const int pos = base + k;
        if (pos >= A.item_cap) break;   // cannot happen: item_cap = ncap (1 + nghost_x)
        // the lower end of copy k, as the scans recompute it
        const double e = __dadd_rn(ext_of(A, i), g.m);
        const double lo = __dsub_rn(__dadd_rn(A.P.x[i], __dmul_rn((double)k, g.lx)), e);
        A.key[pos] = ((uint64_t)b << 32) | quant(lo, g.base, g.scale);
        A.val[pos] = ((uint32_t)i << 3) | (uint32_t)k;
    }
}

// Particle data of the sorted items, gathered once so that the scans read
// neighbouring records instead of scattered particle slots.
struct __align__(16) SweepRec {
    double x, y, z, vx, vy, vz, r;   // the particle's own (unshifted) state
    int id;                          // global id
    uint32_t sc;                     // (slot << 3) | copy
};

__global__ void __launch_bounds__(256) k_sweep_gather(SweepArgs A, const uint32_t* __restrict__ val,
                                                      SweepRec* __restrict__ rec) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int nitem = min(A.ctl->sweep_items, A.item_cap);
    if (k >= nitem) return;
    const uint32_t v = val[k];
    const int i = (int)(v >> 3);
    SweepRec q;
    q.x = A.P.x[i]; q.y = A.P.y[i]; q.z = A.P.z[i];
    q.vx = A.P.vx[i]; q.vy = A.P.vy[i]; q.vz = A.P.vz[i];
    q.r = A.P.r[i];
    q.id = A.P.id[i];
    q.sc = v;
    rec[k] = q;
}

// Straight-line criterion (Sect. 5.3, readings S1/S2) for particle a and the
// image of b (offset o, y velocity offset dvy), in the oracle's operation
// sequence.
__device__ __forceinline__ bool line_hit(const SweepRec& a, const SweepRec& b, double h, double ox,
                                         double oy, double oz, double dvy) {
    const double rx = __dsub_rn(__dadd_rn(b.x, ox), a.x);
    const double ry = __dsub_rn(__dadd_rn(b.y, oy), a.y);
    const double rz = __dsub_rn(__dadd_rn(b.z, oz), a.z);
    const double ux = __dsub_rn(b.vx, a.vx);
    const double uy = __dsub_rn(__dadd_rn(b.vy, dvy), a.vy);
    const double uz = __dsub_rn(b.vz, a.vz);
    const double uu = __dadd_rn(__dadd_rn(__dmul_rn(ux, ux), __dmul_rn(uy, uy)), __dmul_rn(uz, uz));
    const double ru = __dadd_rn(__dadd_rn(__dmul_rn(rx, ux), __dmul_rn(ry, uy)), __dmul_rn(rz, uz));
    double tau = 0.0;
    if (uu > 0.0) {
        tau = __ddiv_rn(-ru, uu);
        if (tau < -h) tau = -h;
        if (tau > h) tau = h;
    }
    const double dx = __dadd_rn(rx, __dmul_rn(ux, tau));
    const double dy = __dadd_rn(ry, __dmul_rn(uy, tau));
    const double dz = __dadd_rn(rz, __dmul_rn(uz, tau));
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    const double s = __dadd_rn(a.r, b.r);
    return d2 < __dmul_rn(s, s);
}

__global__ void __launch_bounds__(128) k_sweep_pairs(SweepArgs A, const SweepRec* __restrict__ rec) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int nitem = min(A.ctl->sweep_items, A.item_cap);
    if (k >= nitem) return;
    const SweepRec Pk = rec[k];
    const int ci = (int)(Pk.sc & 7u);
    const int si = (int)(Pk.sc >> 3);
    const int b = (int)(A.key[k] >> 32);
    const BoxP bp = A.boxes[b];
    const Range g = range_of(A, bp);
    const double hi = __dadd_rn(__dadd_rn(Pk.x, __dmul_rn((double)ci, g.lx)),
                                __dadd_rn(__dadd_rn(__dmul_rn(fabs(Pk.vx), A.h), Pk.r), g.m));
    const uint64_t khi = ((uint64_t)b << 32) | quant(hi, g.base, g.scale);
    // more trajectories cut by the plane than the sweep is meant for (the
    // O(N N_SWEEPL) cost of Sect. 5.3 turning quadratic): report, do not scan
    const int lim = k + 1 + kMaxSweepScan;
    if (lim < nitem && A.key[lim] <= khi) {
        atomicOr(&A.ctl->err, kErrSweepLong);
        return;
    }
    const double s = shear_offset(bp, time_of(A.ctl, A.t0, A.half_dt, A.hs));
    for (int j = k + 1; j < nitem; j++) {
        if (A.key[j] > khi) break;   // at the latest at lim (keys are sorted)
        if (((j - k) & 1023) == 0 && (*(volatile const int*)&A.ctl->err & kErrSweepLong)) break;
        const SweepRec Q = rec[j];
        const int cj = (int)(Q.sc & 7u);
        if ((ci != 0 && cj != 0) || (int)(Q.sc >> 3) == si) continue;
        // image of Q's particle as seen from Pk's, then the canonical orientation
        int gx = cj - ci;
        const bool flip = Q.id < Pk.id;
        if (flip) gx = -gx;
        const SweepRec ra = flip ? Q : Pk;
        const SweepRec rbb = flip ? Pk : Q;
        const double dvy = __dmul_rn(-(double)gx, bp.shear_speed);
        // y extent of the relative motion: |dy(tau)| <= |dy(0)| + |u_y| h for every image
        const double uy = fabs(__dsub_rn(__dadd_rn(rbb.vy, dvy), ra.vy));
        const double ylim = (uy * A.h + (ra.r + rbb.r)) * (1.0 + 1e-12) + g.m;
        const double dyab = rbb.y - ra.y;
        const double gxs = __dmul_rn((double)gx, s);
        for (int gy = -A.ngy; gy <= A.ngy; gy++) {
            const double dy0 = dyab + (__dmul_rn((double)gy, bp.Ly) - gxs);
            if (fabs(dy0) > ylim) continue;
            for (int gz = -A.ngz; gz <= A.ngz; gz++) {
                double ox, oy, oz;
                image_offset(bp, s, gx, gy, gz, ox, oy, oz);
                if (!line_hit(ra, rbb, A.h, ox, oy, oz, dvy)) continue;
                const int code = (gx + 7) | ((gy + 7) << 4) | ((gz + 7) << 8);
                // one atomic per group of lanes that hit together
                cg::coalesced_group grp = cg::coalesced_threads();
                int slot = 0;
                if (grp.thread_rank() == 0) slot = atomicAdd(&A.ctl->pair_count, (int)grp.size());
                slot = grp.shfl(slot, 0) + (int)grp.thread_rank();
                if (slot < A.pair_cap)
                    A.pair_key[slot] = ((uint64_t)ra.id << 36) | ((uint64_t)rbb.id << 12) | (uint64_t)code;
                else
                    atomicOr(&A.ctl->err, kErrPairOverflow);
            }
        }
    }
}

__global__ void k_sweep_reset(Ctl* ctl) {
    ctl->sweep_items = 0;
    ctl->sweep_wbits = 0ull;
}

}  // namespace

void sweep_search(const PSet& P, Ctl* ctl, const BoxP* boxes, const SimC& C, Sweep& S,
                  const Pairs& PR, int half_step_offset, int ncap, cudaStream_t s) {
    if (ncap <= 0) return;
    SweepArgs A;
    A.P = P; A.ctl = ctl; A.boxes = boxes;
    A.key = S.key; A.val = S.val;
    A.pair_key = PR.key; A.pair_cap = PR.cap; A.item_cap = S.cap; A.ncap = ncap; A.nbox = C.nbox;
    A.ngx = C.ngx; A.ngy = C.ngy; A.ngz = C.ngz; A.hs = half_step_offset;
    A.t0 = C.t0; A.half_dt = C.half_dt; A.h = 0.5 * C.dt;
    k_sweep_reset<<<1, 1, 0, s>>>(ctl);
    k_sweep_ext<<<ceil_div(ncap, 256), 256, 0, s>>>(A);
    k_sweep_items<<<ceil_div(ncap, 256), 256, 0, s>>>(A);
    const int key_bits = 32 + S.box_bits;
    const int which = radix_sort(S.key, S.val, S.key_alt, S.val_alt, S.cap, &ctl->sweep_items, key_bits,
                                 nullptr, 0, S.hist, &ctl->err, s);
    if (which == 1) {
        A.key = S.key_alt;
        A.val = S.val_alt;
    }
    SweepRec* rec = static_cast<SweepRec*>(S.rec);
    k_sweep_gather<<<ceil_div(S.cap, 256), 256, 0, s>>>(A, A.val, rec);
    k_sweep_pairs<<<ceil_div(S.cap, 128), 128, 0, s>>>(A, rec);
}

}  // namespace rb
