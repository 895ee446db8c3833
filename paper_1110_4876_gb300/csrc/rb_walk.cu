// rb_walk.cu -- Barnes-Hut gravity walk (Sect. 4.2, Eq. 1) and tree
// collision search (Sect. 5.2, Eq. 3) over the ghost images of Sect. 2.3.
//
// Warp-cooperative stackless walk.  Each warp owns 32 consecutive targets in
// Morton order (spatially close); each lane keeps its own "next entry" in the
// pre-order entry array, exactly as a per-particle stackless walk would.  The
// warp always processes the smallest next entry of its lanes (one __reduce_min
// vote); that entry's record is a broadcast load, and only the lanes whose
// next entry it is evaluate their own opening test.  Every lane therefore
// accepts, opens and interacts with exactly the cells of its own walk, so the
// accepted cell sets equal the oracle's; lanes skip the entries their own
// walk does not visit.
//
// FP32 walk: the target point and every centre of mass are hi/lo float pairs,
// so (hi_c - hi_p) + (lo_c - lo_p) keeps ~1e-7 relative accuracy even for
// neighbours a metre apart in a 2 km box.  An opening test whose two sides
// differ by less than 1e-5 relative is decided again in FP64 on the FP64
// centre of mass, with the same operation sequence as the oracle.
#include <cfloat>
#include <mutex>
#include <vector>

#include "rb_internal.cuh"
#include "rb_mlp.cuh"

namespace rb {
namespace {

constexpr unsigned kFull = 0xffffffffu;

struct GravArgs {
    const double *x, *y, *z;
    const int32_t* box;
    Rec4 ra, rb, rq0, rq1, rc_hi, rc_lo;
    const double4_32a *d_a, *d_q0, *d_q1, *d_c;
    const int32_t *e_skip, *leaf_of, *box_root;
    const uint32_t* order;      // tile order of the targets (nullptr: Morton order of the slots)
    const int32_t* e_child;     // per cell entry: child entry of each octant (group walk)
    const uint32_t* e_cmask;    // per cell entry: octants holding a child (0: depth-21 group)
    const BoxP* boxes;
    Ctl* ctl;
    WalkOut out;
    int ncap;
    int ngx, ngy, ngz;
    int half_step_offset;
    double G, theta2, soft2, t0, half_dt;
    float soft2f;
    // recording of accepted cells in the band w/R > theta_lo (learned mode)
    uint64_t* req;
    int* req_count;
    int req_cap;
    float band_scale;   // (theta_lo / theta)^2: band iff (w/theta)^2 > band_scale R^2
    uint32_t thresh;    // keep a request when its hash < thresh (0xffffffff: all)
    uint32_t seed;
    // learned walk: cell particle counts (an input of the network) and weights
    const int32_t* e_count;
    const mlp::Packed* wpk;
    int ecap;   // entry capacity (every entry index below it is readable)
    const ImgTab* img;   // [box][image] offsets at the time of this walk
    int nimg;
    int32_t* tq;         // tile queues (emptied by the image-table launch)
    int nq;
};

__device__ __forceinline__ double4_32a ld_d4(const double4_32a* p) { return *p; }

// Counter-based hash of a (target, cell, image) request for subsampling.
__device__ __forceinline__ uint32_t req_hash(uint32_t slot, uint32_t entry, uint32_t code,
                                             uint32_t seed) {
    uint32_t h = slot * 0x9E3779B1u ^ (entry + 0x7F4A7C15u) * 0x85EBCA77u ^ code * 0xC2B2AE3Du ^ seed;
    h ^= h >> 16;
    h *= 0x7FEB352Du;
    h ^= h >> 15;
    h *= 0x846CA68Bu;
    h ^= h >> 16;
    return h;
}

// Opening test in FP64, operation for operation as the oracle evaluates it.
__device__ __forceinline__ bool mac64(const double4_32a& a, double theta2, double tx, double ty,
                                      double tz) {
    const double dx = __dsub_rn(a.x, tx), dy = __dsub_rn(a.y, ty), dz = __dsub_rn(a.z, tz);
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return a.w < __dmul_rn(theta2, r2);
}

// 1/sqrt(x) from the hardware estimate plus one Newton step
// y' = y (3/2 - x y^2 / 2), which roughly halves its relative error.
__device__ __forceinline__ float rsqrt_nr(float x) {
    const float y = rsqrtf(x);
    return y * fmaf((-0.5f * x) * y, y, 1.5f);
}

// Compensated (Kahan) accumulation: in a sheet the net force is often a
// small remainder of much larger cancelling terms, and a plain FP32 running
// sum loses ~1e-5 of it.  The walk sums terms plainly over at most 16 warp
// iterations and adds those short partial sums into Kahan sums, whose
// running compensation c keeps the lost low-order bits.
__device__ __forceinline__ void kadd(float& s, float& c, float t) {
    const float y = t - c;
    const float u = s + y;
    c = (u - s) - y;
    s = u;
}

// Tile scheduling of the walks: queue q owns tiles [b_q, b_{q+1}) with
// b_q = floor(q T / nq) of the T tiles of 32 consecutive targets.
__device__ __forceinline__ int tile_begin(int q, int ntile, int nq) {
    return (int)(((long long)q * ntile) / nq);
}

__device__ __forceinline__ int sm_queue(int nq) {
    unsigned sm;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
    return (int)(sm % (unsigned)nq);
}

// Slot of the k-th target in tile order.
__device__ __forceinline__ int tile_slot(const uint32_t* order, int k) {
    return order ? (int)__ldg(&order[k]) : k;
}

// The warp's next tile, or -1 when every queue is empty: its own SM's queue
// first, then the following queues (32 probed per vote).  Warp-uniform.
__device__ __noinline__ int next_tile(int32_t* tq, int nq, int q, int ntile) {
    const int lane = threadIdx.x & 31;
    int t = -1;
    if (lane == 0) {
        const int b = tile_begin(q, ntile, nq);
        const int k = atomicAdd(&tq[q * kTileQStride], 1);
        if (k < tile_begin(q + 1, ntile, nq) - b) t = b + k;
    }
    t = __shfl_sync(kFull, t, 0);
    if (t >= 0) return t;
    for (int k0 = 1; k0 < nq; k0 += 32) {
        const int off = k0 + lane;
        int qq = q + off;
        if (qq >= nq) qq -= nq;
        int b = 0, len = 0;
        bool avail = false;
        if (off < nq) {
            b = tile_begin(qq, ntile, nq);
            len = tile_begin(qq + 1, ntile, nq) - b;
            avail = __ldcg(&tq[qq * kTileQStride]) < len;
        }
        for (unsigned m = __ballot_sync(kFull, avail); m; m &= m - 1) {
            const int src = __ffs(m) - 1;
            int got = -1;
            if (lane == src) {
                const int k = atomicAdd(&tq[qq * kTileQStride], 1);
                if (k < len) got = b + k;
            }
            got = __shfl_sync(kFull, got, src);
            if (got >= 0) return got;
        }
    }
    return -1;
}

// Ghost-image table of the walk or search time: one thread per (box, image),
// images in the kernels' loop order (gx outermost, gz innermost), for boxes
// 0 .. nbox (row nbox, a copy of box 0's, is read by removed particles, which
// search nothing).  Threads below nq * kTileQStride also empty the tile
// queues.
__global__ void k_img_table(const BoxP* __restrict__ boxes, const Ctl* __restrict__ ctl, double t0,
                            double half_dt, int hs, int nbox, int ngx, int ngy, int ngz,
                            ImgTab* __restrict__ tab, int32_t* __restrict__ tq, int nqw) {
    const int ny = 2 * ngy + 1, nz = 2 * ngz + 1;
    const int nimg = (2 * ngx + 1) * ny * nz;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nqw) tq[k] = 0;
    if (k >= (nbox + 1) * nimg) return;
    const int b = k / nimg, g = k % nimg;
    const int gz = g % nz - ngz, gy = (g / nz) % ny - ngy, gx = g / (ny * nz) - ngx;
    const BoxP bp = boxes[b < nbox ? b : 0];
    const double s = shear_offset(bp, time_of(ctl, t0, half_dt, hs));
    ImgTab T;
    image_offset(bp, s, gx, gy, gz, T.ox, T.oy, T.oz);
    T.dvy = __dmul_rn(-(double)gx, bp.shear_speed);
    const float hx = __double2float_rn(T.ox), hy = __double2float_rn(T.oy), hz = __double2float_rn(T.oz);
    T.hi = make_float4(hx, hy, hz, 0.f);
    T.lo = make_float4(__double2float_rn(T.ox - (double)hx), __double2float_rn(T.oy - (double)hy),
                       __double2float_rn(T.oz - (double)hz), 0.f);
    tab[k] = T;
}

// t = p - o for hi/lo float pairs: the rounding error of ph - oh is kept
// (Knuth's two-sum) and the low parts are subtracted, so t is good to about
// 2^-45 of |p| without any FP64 arithmetic.
__device__ __forceinline__ void sub_hilo(float ph, float pl, float oh, float ol, float& th, float& tl) {
    const float s = ph - oh;
    const float bb = s - ph;
    const float e = (ph - (s - bb)) + (-oh - bb);
    th = s;
    tl = e + (pl - ol);
}

__device__ __forceinline__ void split_d(double v, float& hi, float& lo) {
    hi = __double2float_rn(v);
    lo = __double2float_rn(v - (double)hi);
}

// Is the target point inside the closed cube of a cell (FP64, exact sequence)?
__device__ __forceinline__ bool inside64(const double4_32a& c, double tx, double ty, double tz) {
    return c.x <= tx && tx <= __dadd_rn(c.x, c.w) && c.y <= ty && ty <= __dadd_rn(c.y, c.w) &&
           c.z <= tz && tz <= __dadd_rn(c.z, c.w);
}

// Per-warp queue of the learned walk: accepted band cells waiting for the
// network, which runs on 16 of them at a time (one m16 tile).
struct LearnQ {
    __nv_bfloat16 X[48][16];   // network inputs (columns 12..15 zero)
    float unit[48];            // M / R^2 (G is applied with the walk's sums)
    int own[48];               // lane whose sums receive the output
    float Y[16][4];            // outputs of the tile being applied
};

// Rows r0 .. r0 + 15 of the queue through the network; unit * output is
// added to the owning lanes' partial sums.  Warp-synchronous.
__device__ __forceinline__ void learn_flush(LearnQ& Q, const mlp::Packed& w, int r0, int lane,
                                            float& fx, float& fy, float& fz) {
    __syncwarp();
    float out[4];
    mlp::forward_packed(w, &Q.X[r0][0], out);
    const int g = lane >> 2, q = lane & 3;
    if (q < 2) {
        Q.Y[g][2 * q] = out[0];
        Q.Y[g][2 * q + 1] = out[1];
        Q.Y[g + 8][2 * q] = out[2];
        Q.Y[g + 8][2 * q + 1] = out[3];
    }
    __syncwarp();
#pragma unroll 4
    for (int k = 0; k < 16; k++)
        if (Q.own[r0 + k] == lane) {
            const float u = Q.unit[r0 + k];
            fx += u * Q.Y[k][0];
            fy += u * Q.Y[k][1];
            fz += u * Q.Y[k][2];
        }
    __syncwarp();
}

// kOne: a single box, so every lane's walk ends at the same entry and no
// lane can run into another box's tree.
template <bool kQuad, bool kInside, bool kPot, bool kSoft, bool kRecord, bool kLearn, bool kOne = false>
__device__ __forceinline__ void walk32(const GravArgs& A, LearnQ* LQ, const mlp::Packed* W, int wbase,
                                       int n) {
    const int lane = threadIdx.x & 31;
    const bool valid = wbase + lane < n;
    const int ii = tile_slot(A.order, valid ? wbase + lane : n - 1);
    const int i = ii;   // the target's slot
    const int root = A.box_root[A.box[ii]];
    const int wend = root >= 0 ? A.e_skip[root] : 0;   // end of this box's tree
    const int self_leaf = A.leaf_of[ii];
    // the FP64 target point of the current image: read only by the rare FP64
    // re-decisions, so it lives in shared memory rather than in registers
    // the target particle as hi/lo floats; each image's offset comes from the
    // image table, so no FP64 arithmetic is needed per image
    float phx, plx, phy, ply, phz, plz;
    split_d(A.x[ii], phx, plx);
    split_d(A.y[ii], phy, ply);
    split_d(A.z[ii], phz, plz);
    const ImgTab* itab = A.img + (size_t)A.box[ii] * A.nimg;
    int gi = 0;
    double pot = 0.0;
    float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;  // sums + compensation
    int ncell = 0, nleaf = 0, nmac = 0, nrecheck = 0, ncorr = 0;
    int iters = 0;   // entries processed by the warp (warp-uniform)
    int qn = 0;   // kLearn: rows waiting in this warp's queue (warp-uniform)
    for (int gx = -A.ngx; gx <= A.ngx; gx++)
        for (int gy = -A.ngy; gy <= A.ngy; gy++)
            for (int gz = -A.ngz; gz <= A.ngz; gz++, gi++) {
                float thx, thy, thz, tlx, tly, tlz;
                {
                    const float4 oh = itab[gi].hi, ol = itab[gi].lo;
                    sub_hilo(phx, plx, oh.x, ol.x, thx, tlx);
                    sub_hilo(phy, ply, oh.y, ol.y, thy, tly);
                    sub_hilo(phz, plz, oh.z, ol.z, thz, tlz);
                }
                // negated target (x, y) pairs for the packed FP32 adds (two
                // adds per instruction on sm_103a, and the walk is bound by
                // instruction issue): a - t = a + (-t) exactly, so they give
                // the scalar differences bit for bit
                const float2 nth = make_float2(-thx, -thy), ntl = make_float2(-tlx, -tly);
                const float2 ntz = make_float2(-thz, -tlz);   // z: (hi, lo) of the target
                const int self = (gx == 0 && gy == 0 && gz == 0) ? self_leaf : -1;
                int next = (valid && root >= 0) ? root : kEnd;
                float fx = 0.f, fy = 0.f, fz = 0.f, fp = 0.f;   // sums of the last <= 16 iterations
                int it = 0;           // entries processed (warp-uniform)
                bool rec = false;     // kRecord: this lane accepted a band cell this iteration
                uint64_t rkey = 0;
                bool want = false;    // kLearn: this lane accepted a band cell this iteration
                float fin[12], funit = 0.f;
                // one entry of the union walk; false when every lane is done
                auto step = [&]() -> bool {
                    if (!kOne && next >= wend) next = kEnd;
                    const int e = (int)__reduce_min_sync(kFull, (unsigned)next);
                    if (kOne ? e >= wend : e == kEnd) return false;
                    const float4 ra = __ldg(&A.ra[e]);
                    const float4 rb = __ldg(&A.rb[e]);
                    const bool act = next == e;
                    const float2 dxy = __fadd2_rn(__fadd2_rn(make_float2(ra.x, ra.y), nth),
                                                  __fadd2_rn(make_float2(rb.x, rb.y), ntl));
                    const float dx = dxy.x, dy = dxy.y;
                    const float2 zz = __fadd2_rn(make_float2(ra.z, ra.w), ntz);
                    const float dz = zz.x + zz.y;
                    const float crit = rb.z;   // leaf: -m; cell: (w / theta)^2
                    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                    if (__float_as_int(crit) < 0) {
                        // particle leaf: exact term of Eq. 1
                        if (act) {
                            if (e != self) {
                                const float m = -crit;
                                const float inv = rsqrt_nr(kSoft ? r2 + A.soft2f : r2);
                                const float f = m * (inv * inv * inv);
                                fx = fmaf(f, dx, fx);
                                fy = fmaf(f, dy, fy);
                                fz = fmaf(f, dz, fz);
                                if (kPot) fp = fmaf(-m, inv, fp);
                                nleaf++;
                            }
                            next = e + 1;
                        }
                    } else if (act) {
                        nmac++;
                        bool acc = crit < r2;
                        if (fabsf(crit - r2) <= 1e-5f * r2) {
                            // the FP64 target point x - o, as the oracle forms it
                            acc = mac64(ld_d4(&A.d_a[e]), A.theta2, __dsub_rn(A.x[ii], itab[gi].ox),
                                        __dsub_rn(A.y[ii], itab[gi].oy), __dsub_rn(A.z[ii], itab[gi].oz));
                            nrecheck++;
                        }
                        if (kInside && acc) {
                            const float4 ch = __ldg(&A.rc_hi[e]);
                            const float4 cl = __ldg(&A.rc_lo[e]);
                            const float ux = (thx - ch.x) + (tlx - cl.x);
                            const float uy = (thy - ch.y) + (tly - cl.y);
                            const float uz = (thz - ch.z) + (tlz - cl.z);
                            const float w = ch.w, tol = 1e-5f * ch.w;
                            const float mx = fminf(fminf(ux, w - ux), fminf(fminf(uy, w - uy), fminf(uz, w - uz)));
                            if (fabsf(mx) <= tol) {
                                acc = !inside64(ld_d4(&A.d_c[e]), __dsub_rn(A.x[ii], itab[gi].ox),
                                                __dsub_rn(A.y[ii], itab[gi].oy),
                                                __dsub_rn(A.z[ii], itab[gi].oz));
                                nrecheck++;
                            } else if (mx > 0.f) {
                                acc = false;
                            }
                        }
                        if (acc) {
                            const float4 q0 = __ldg(&A.rq0[e]);
                            const float4 q1 = __ldg(&A.rq1[e]);
                            // monopole and quadrupole (reading R3) with the radial
                            // factors merged: a = (M/R^3 + 2.5 dQd/R^7) d - Q d/R^5
                            const float inv = rsqrt_nr(r2);
                            const float inv2 = inv * inv;
                            const float invs = kSoft ? rsqrt_nr(r2 + A.soft2f) : inv;
                            float fc = q0.x * (kSoft ? invs * invs * invs : inv2 * inv);
                            if (kPot) fp = fmaf(-q0.x, invs, fp);
                            if (kQuad) {
                                const float qx = fmaf(q1.y, dz, fmaf(q1.x, dy, q0.y * dx));
                                const float qy = fmaf(q1.z, dz, fmaf(q0.z, dy, q1.x * dx));
                                const float qz = fmaf(q0.w, dz, fmaf(q1.z, dy, q1.y * dx));
                                const float dqd = fmaf(dz, qz, fmaf(dy, qy, dx * qx));
                                const float inv5 = inv2 * inv2 * inv;
                                fc = fmaf(2.5f, dqd * (inv5 * inv2), fc);
                                fx = fmaf(-inv5, qx, fx);
                                fy = fmaf(-inv5, qy, fy);
                                fz = fmaf(-inv5, qz, fz);
                                if (kPot) fp = fmaf(-0.5f * dqd, inv5, fp);
                            }
                            fx = fmaf(fc, dx, fx);
                            fy = fmaf(fc, dy, fy);
                            fz = fmaf(fc, dz, fz);
                            ncell++;
                            next = __float_as_int(rb.w);
                            if (kLearn && crit > A.band_scale * r2) {
                                // network inputs (the oracle's definition, in FP32 from the
                                // walk records): r = p - com = -d
                                const float4 ch = __ldg(&A.rc_hi[e]);
                                const float4 cl = __ldg(&A.rc_lo[e]);
                                const float w = ch.w, rw = 1.f / w;
                                const float hx = -dx * inv, hy = -dy * inv, hz = -dz * inv;
                                const float sc = rw * rw / q0.x;
                                const float qxx = q0.y * sc, qyy = q0.z * sc, qzz = q0.w * sc;
                                const float qxy = q1.x * sc, qxz = q1.y * sc, qyz = q1.z * sc;
                                const float ux = qxx * hx + qxy * hy + qxz * hz;
                                const float uy = qxy * hx + qyy * hy + qyz * hz;
                                const float uz = qxz * hx + qyz * hy + qzz * hz;
                                fin[0] = hx; fin[1] = hy; fin[2] = hz;
                                fin[3] = w * inv;
                                fin[4] = __log2f((float)__ldg(&A.e_count[e])) * 0.30102999566f;
                                fin[5] = ((ra.x - ch.x) + (rb.x - cl.x)) * rw - 0.5f;
                                fin[6] = ((ra.y - ch.y) + (rb.y - cl.y)) * rw - 0.5f;
                                fin[7] = ((ra.z - ch.z) + (ra.w - cl.z)) * rw - 0.5f;
                                fin[8] = hx * ux + hy * uy + hz * uz;
                                fin[9] = sqrtf(ux * ux + uy * uy + uz * uz);
                                fin[10] = qxx * qxx + qyy * qyy + qzz * qzz +
                                          2.f * (qxy * qxy + qxz * qxz + qyz * qyz);
                                fin[11] = qxx * (qyy * qzz - qyz * qyz) - qxy * (qxy * qzz - qyz * qxz) +
                                          qxz * (qxy * qyz - qyy * qxz);
                                funit = q0.x * inv2;
                                want = true;
                            }
                            if (kRecord && crit > A.band_scale * r2) {
                                const uint32_t code = (gx + 7) | ((gy + 7) << 4) | ((gz + 7) << 8);
                                rec = A.thresh == 0xffffffffu ||
                                      req_hash((uint32_t)i, (uint32_t)e, code, A.seed) < A.thresh;
                                if (rec)
                                    rkey = ((uint64_t)i << 40) | ((uint64_t)code << 28) | (uint64_t)e;
                            }
                        } else {
                            next = e + 1;
                        }
                    }
                    if (kRecord) {
                        // accepted band cells of this iteration, appended warp by warp
                        const unsigned m = __ballot_sync(kFull, rec);
                        if (m) {
                            const int leader = __ffs(m) - 1;
                            int pos = 0;
                            if (lane == leader) pos = atomicAdd(A.req_count, __popc(m));
                            pos = __shfl_sync(kFull, pos, leader) + __popc(m & ((1u << lane) - 1u));
                            if (rec && pos < A.req_cap) A.req[pos] = rkey;
                        }
                        rec = false;
                    }
                    if (kLearn) {
                        // band cells of this iteration join the warp's queue; full
                        // tiles of 16 go through the network
                        const unsigned m = __ballot_sync(kFull, want);
                        if (m) {
                            if (want) {
                                const int pos = qn + __popc(m & ((1u << lane) - 1u));
                                uint4 lo, hi;
                                lo.x = mlp::pack2(fin[0], fin[1]);
                                lo.y = mlp::pack2(fin[2], fin[3]);
                                lo.z = mlp::pack2(fin[4], fin[5]);
                                lo.w = mlp::pack2(fin[6], fin[7]);
                                hi.x = mlp::pack2(fin[8], fin[9]);
                                hi.y = mlp::pack2(fin[10], fin[11]);
                                hi.z = 0u;
                                hi.w = 0u;
                                reinterpret_cast<uint4*>(&LQ->X[pos][0])[0] = lo;
                                reinterpret_cast<uint4*>(&LQ->X[pos][0])[1] = hi;
                                LQ->unit[pos] = funit;
                                LQ->own[pos] = lane;
                                ncorr++;
                            }
                            qn += __popc(m);
                            while (qn >= 16) {
                                qn -= 16;
                                learn_flush(*LQ, *W, qn, lane, fx, fy, fz);
                            }
                        }
                        want = false;
                    }
                    return true;
                };
                // two entries per pass (one with the network or the band
                // record inside, whose code is large); the warp-uniform flush
                // into the compensated sums every 16 entries
                for (;;) {
                    if (it != 0 && (it & 15) == 0) {
                        kadd(sx, cx, fx);
                        kadd(sy, cy, fy);
                        kadd(sz, cz, fz);
                        fx = fy = fz = 0.f;
                    }
                    if (!step()) break;
                    if (kLearn || kRecord) {
                        it += 1;
                        continue;
                    }
                    if (!step()) {
                        it += 1;
                        break;
                    }
                    it += 2;
                }
                kadd(sx, cx, fx);
                kadd(sy, cy, fy);
                kadd(sz, cz, fz);
                pot += (double)fp;
                iters += it;
            }
    if (kLearn && qn > 0) {
        // the last partial tile: empty rows have zero inputs and no owner
        if (lane >= qn && lane < 16) {
            reinterpret_cast<uint4*>(&LQ->X[lane][0])[0] = make_uint4(0u, 0u, 0u, 0u);
            reinterpret_cast<uint4*>(&LQ->X[lane][0])[1] = make_uint4(0u, 0u, 0u, 0u);
            LQ->unit[lane] = 0.f;
            LQ->own[lane] = -1;
        }
        float fx = 0.f, fy = 0.f, fz = 0.f;
        learn_flush(*LQ, *W, 0, lane, fx, fy, fz);
        kadd(sx, cx, fx);
        kadd(sy, cy, fy);
        kadd(sz, cz, fz);
    }
    if (valid) {
        A.out.ax[i] = A.G * ((double)sx - (double)cx);
        A.out.ay[i] = A.G * ((double)sy - (double)cy);
        A.out.az[i] = A.G * ((double)sz - (double)cz);
        if (kPot) A.out.phi[i] = A.G * pot;
        if (A.out.ncell) {
            A.out.ncell[i] = ncell;
            A.out.nleaf[i] = nleaf;
            A.out.nmac[i] = nmac;
        }
    }
    // warp totals of the counters
    unsigned long long c0 = valid ? ncell : 0, c1 = valid ? nleaf : 0, c2 = valid ? nmac : 0,
                       c3 = valid ? nrecheck : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c0 += __shfl_down_sync(kFull, c0, o);
        c1 += __shfl_down_sync(kFull, c1, o);
        c2 += __shfl_down_sync(kFull, c2, o);
        c3 += __shfl_down_sync(kFull, c3, o);
    }
    if (lane == 0) {
        atomicAdd(&A.ctl->n_cell, c0);
        atomicAdd(&A.ctl->n_leaf, c1);
        atomicAdd(&A.ctl->n_mac, c2);
        atomicAdd(&A.ctl->n_recheck, c3);
        atomicAdd(&A.ctl->n_iter, (unsigned long long)iters);
    }
    if (kLearn) {
        int c4 = ncorr;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c4 += __shfl_down_sync(kFull, c4, o);
        if (lane == 0) atomicAdd(&A.ctl->req_count, c4);
    }
}

template <bool kQuad, bool kInside, bool kPot, bool kSoft, bool kRecord = false, bool kOne = false>
__global__ void __launch_bounds__(kMaxWalkBlock, 4) k_walk32(GravArgs A) {
    const int n = min(A.ctl->n_live, A.ncap);
    const int ntile = (n + 31) >> 5, q = sm_queue(A.nq);
    for (int t = next_tile(A.tq, A.nq, q, ntile); t >= 0; t = next_tile(A.tq, A.nq, q, ntile))
        walk32<kQuad, kInside, kPot, kSoft, kRecord, false, kOne>(A, nullptr, nullptr, t << 5, n);
}

// ---------------------------------------------------------------------------
// Group walk (FP32, plain): exact per-target accepted sets, far field decided
// once per warp.
//
// For each ghost image the warp first walks the tree as a group: the lanes
// take up to 32 frontier cells at a time and test each against the bounding
// box of the warp's 32 target points.  A cell that every target point
// provably accepts (its opening test w < theta R holds for the box's nearest
// point with a 1e-4 margin, so each lane's own FP32 test would accept it
// outside the FP64 guard band) goes to the warp's interaction list; a cell
// that every target provably opens (the test fails for the box's farthest
// point) has its children pushed to the frontier; a leaf reached this way is
// an exact term for every target but its own particle.  Any other cell is
// "mixed": its subtree is walked afterwards target by target with the same
// per-lane opening test (FP32, re-decided in FP64 near the threshold, inside
// rule) as the union walk, so each target visits exactly the cells its own
// Barnes-Hut walk visits (Sect. 4.2) and the accepted sets equal the oracle's.
//
// The list is evaluated by all 32 lanes with broadcast record loads; the
// mixed subtrees are walked by subgroups of kS lanes, each subgroup taking
// the smallest next entry of its own lanes (a union walk over kS targets, far
// fewer idle lanes than over 32), the subgroups advancing through the mixed
// list independently.
constexpr int kGFront = 192;   // frontier cells per warp
constexpr int kGList = 64;     // accepted list per warp (evaluated when nearly full)
constexpr int kGMix = 96;      // mixed subtrees per warp (walked when nearly full)

struct GroupSmem {
    float4 rec[kGList][4];   // accepted list: the entries' records ra, rb, rq0, rq1
    int front[kGFront];
    int2 mix[kGMix];         // (entry, image)
    float box[10];           // current image: bounding box (x0 x1 y0 y1 z0 z1), extent, reference point
};

// Per-lane state of the group walk of one tile.
struct GLane {
    float sx, sy, sz, cx, cy, cz;         // Kahan sums and their compensation
    float fx, fy, fz;                     // plain sums of the last <= 16 terms
    int ncell, nleaf, nmac, nrecheck;
    int iters;                            // warp iterations (warp-uniform)
    int fcount;                           // terms since the last flush (warp-uniform)
};

__device__ __forceinline__ void glane_flush(GLane& L) {
    kadd(L.sx, L.cx, L.fx);
    kadd(L.sy, L.cy, L.fy);
    kadd(L.sz, L.cz, L.fz);
    L.fx = L.fy = L.fz = 0.f;
}

__device__ __forceinline__ void glane_count(GLane& L) {
    if (++L.fcount == 16) {
        glane_flush(L);
        L.fcount = 0;
    }
}

// Monopole + quadrupole term of an accepted cell (reading R3), the same
// arithmetic as the union walk's; a particle leaf is the cell with Q = 0.
template <bool kQuad, bool kSoft>
__device__ __forceinline__ void cell_term(float dx, float dy, float dz, float r2, const float4& q0,
                                          const float4& q1, float soft2f, float& fx, float& fy,
                                          float& fz) {
    const float inv = rsqrt_nr(r2);
    const float inv2 = inv * inv;
    const float invs = kSoft ? rsqrt_nr(r2 + soft2f) : inv;
    float fc = q0.x * (kSoft ? invs * invs * invs : inv2 * inv);
    if (kQuad) {
        const float qx = fmaf(q1.y, dz, fmaf(q1.x, dy, q0.y * dx));
        const float qy = fmaf(q1.z, dz, fmaf(q0.z, dy, q1.x * dx));
        const float qz = fmaf(q0.w, dz, fmaf(q1.z, dy, q1.y * dx));
        const float dqd = fmaf(dz, qz, fmaf(dy, qy, dx * qx));
        const float inv5 = inv2 * inv2 * inv;
        fc = fmaf(2.5f, dqd * (inv5 * inv2), fc);
        fx = fmaf(-inv5, qx, fx);
        fy = fmaf(-inv5, qy, fy);
        fz = fmaf(-inv5, qz, fz);
    }
    fx = fmaf(fc, dx, fx);
    fy = fmaf(fc, dy, fy);
    fz = fmaf(fc, dz, fz);
}

// Record minus target for the negated target point (nxy: x, y hi; lxy: x, y
// lo; nz: z hi, lo).
__device__ __forceinline__ void rec_diff(const float4& ra, const float4& rb, float2 nxy, float2 lxy,
                                         float2 nz, float& dx, float& dy, float& dz, float& r2) {
    const float2 dxy = __fadd2_rn(__fadd2_rn(make_float2(ra.x, ra.y), nxy),
                                  __fadd2_rn(make_float2(rb.x, rb.y), lxy));
    dx = dxy.x;
    dy = dxy.y;
    const float2 zz = __fadd2_rn(make_float2(ra.z, ra.w), nz);
    dz = zz.x + zz.y;
    r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}

// The negated target point x - o of image img as hi/lo floats, formed from
// the particle's FP64 position and the image table's hi/lo offset.
__device__ __forceinline__ void neg_target(const GravArgs& A, int ii, const ImgTab& T, float2& nxy,
                                           float2& lxy, float2& nz) {
    float ph, pl, th, tl, th2, tl2, th3, tl3;
    split_d(A.x[ii], ph, pl);
    sub_hilo(ph, pl, T.hi.x, T.lo.x, th, tl);
    split_d(A.y[ii], ph, pl);
    sub_hilo(ph, pl, T.hi.y, T.lo.y, th2, tl2);
    split_d(A.z[ii], ph, pl);
    sub_hilo(ph, pl, T.hi.z, T.lo.z, th3, tl3);
    nxy = make_float2(-th, -th2);
    lxy = make_float2(-tl, -tl2);
    nz = make_float2(-th3, -tl3);
}

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// All 32 lanes evaluate the staged records rec[0 .. lc) for their own
// target point; `self` is this lane's own leaf in the central image (else
// -1).  A leaf's record holds -m and its entry + 1 in rb.z and rb.w.
template <bool kQuad, bool kSoft>
__device__ __forceinline__ void eval_list(const GravArgs& A, const float4 (*rec)[4], int lc, int ii,
                                          const ImgTab& T, int self, GLane& L) {
    float2 nxy, lxy, nz;
    neg_target(A, ii, T, nxy, lxy, nz);
    for (int j = 0; j < lc; j++) {
        const float4 ra = rec[j][0];
        const float4 rb = rec[j][1];
        float dx, dy, dz, r2;
        rec_diff(ra, rb, nxy, lxy, nz, dx, dy, dz, r2);
        const float crit = rb.z;
        if (__float_as_int(crit) < 0) {
            // particle leaf reached through cells every target opened
            if (__float_as_int(rb.w) - 1 != self) {
                const float m = -crit;
                const float inv = rsqrt_nr(kSoft ? r2 + A.soft2f : r2);
                const float f = m * (inv * inv * inv);
                L.fx = fmaf(f, dx, L.fx);
                L.fy = fmaf(f, dy, L.fy);
                L.fz = fmaf(f, dz, L.fz);
                L.nleaf++;
            }
        } else {
            cell_term<kQuad, kSoft>(dx, dy, dz, r2, rec[j][2], rec[j][3], A.soft2f, L.fx, L.fy, L.fz);
        }
        glane_count(L);
    }
    L.iters += lc;
}

// The per-target walks of the mixed subtrees mix[0 .. mc), by subgroups of
// kS lanes.  Each subgroup walks every subtree for its own lanes: the union
// of its lanes' stackless walks from the subtree's root to its skip entry,
// with the union walk's per-lane opening test.
template <bool kQuad, bool kInside, bool kSoft, int kS>
__device__ __forceinline__ void mixed_walks(const GravArgs& A, const int2* mix, int mc, const ImgTab* itab,
                                            int ii, int self_leaf, int gcentre, GLane& L) {
    int mi = -1, endc = 0, next = kEnd, img = -1, self = -1;
    float2 nxy = make_float2(0.f, 0.f), lxy = nxy, nz = nxy;
    for (;;) {
        int e = next;
#pragma unroll
        for (int o = 1; o < kS; o <<= 1) e = min(e, __shfl_xor_sync(kFull, e, o));
        if (e >= endc) {
            // this subgroup is done with its subtree: take the next one
            ++mi;
            if (mi < mc) {
                const int2 m = mix[mi];
                e = m.x;
                next = m.x;
                endc = __ldg(&A.e_skip[m.x]);
                if (m.y != img) {
                    img = m.y;
                    neg_target(A, ii, itab[img], nxy, lxy, nz);
                    self = img == gcentre ? self_leaf : -1;
                }
            } else {
                e = kEnd;
                endc = kEnd;
                next = kEnd;
                mi = mc;
            }
        }
        if (__all_sync(kFull, e == kEnd)) break;
        if (e != kEnd && e >= A.ecap) {
            // cannot happen for a well-formed tree: record it and stop
            atomicOr(&A.ctl->err, kErrWalk);
            e = kEnd;
            endc = kEnd;
            next = kEnd;
            mi = mc;
        }
        if (e != kEnd) {
            const float4 ra = __ldg(&A.ra[e]);
            const float4 rb = __ldg(&A.rb[e]);
            float dx, dy, dz, r2;
            rec_diff(ra, rb, nxy, lxy, nz, dx, dy, dz, r2);
            const float crit = rb.z;
            const bool leaf = __float_as_int(crit) < 0;
            bool acc = false;
            if (next == e) {
                if (leaf) {
                    acc = e != self;
                    if (acc) L.nleaf++;
                    next = e + 1;
                } else {
                    L.nmac++;
                    acc = crit < r2;
                    if (fabsf(crit - r2) <= 1e-5f * r2) {
                        // the FP64 target point x - o, as the oracle forms it
                        acc = mac64(ld_d4(&A.d_a[e]), A.theta2, __dsub_rn(A.x[ii], itab[img].ox),
                                    __dsub_rn(A.y[ii], itab[img].oy), __dsub_rn(A.z[ii], itab[img].oz));
                        L.nrecheck++;
                    }
                    if (kInside && acc) {
                        const float4 ch = __ldg(&A.rc_hi[e]);
                        const float4 cl = __ldg(&A.rc_lo[e]);
                        const float ux = (-nxy.x - ch.x) + (-lxy.x - cl.x);
                        const float uy = (-nxy.y - ch.y) + (-lxy.y - cl.y);
                        const float uz = (-nz.x - ch.z) + (-nz.y - cl.z);
                        const float w = ch.w, tol = 1e-5f * ch.w;
                        const float mx = fminf(fminf(ux, w - ux), fminf(fminf(uy, w - uy), fminf(uz, w - uz)));
                        if (fabsf(mx) <= tol) {
                            acc = !inside64(ld_d4(&A.d_c[e]), __dsub_rn(A.x[ii], itab[img].ox),
                                            __dsub_rn(A.y[ii], itab[img].oy),
                                            __dsub_rn(A.z[ii], itab[img].oz));
                            L.nrecheck++;
                        } else if (mx > 0.f) {
                            acc = false;
                        }
                    }
                    if (acc) {
                        L.ncell++;
                        next = __float_as_int(rb.w);
                    } else {
                        next = e + 1;
                    }
                }
            }
            if (acc) {
                float4 q0, q1;
                if (leaf) {
                    q0 = make_float4(-crit, 0.f, 0.f, 0.f);
                    q1 = make_float4(0.f, 0.f, 0.f, 0.f);
                } else {
                    q0 = __ldg(&A.rq0[e]);
                    q1 = __ldg(&A.rq1[e]);
                }
                cell_term<kQuad, kSoft>(dx, dy, dz, r2, q0, q1, A.soft2f, L.fx, L.fy, L.fz);
            }
        }
        L.iters++;
        glane_count(L);
    }
}

// One tile of 32 consecutive targets, all in one box.  Images are taken in
// turn; each image's group walk fills the list (evaluated when nearly full
// and when the image is done) and the mixed list (walked when nearly full
// and after the last image).
template <bool kQuad, bool kInside, bool kSoft, int kS>
__device__ __forceinline__ void walk32g(const GravArgs& A, GroupSmem& G, int wbase, int n) {
    const int lane = threadIdx.x & 31;
    const bool valid = wbase + lane < n;
    const int ii = tile_slot(A.order, valid ? wbase + lane : n - 1);
    const int i = ii;   // the target's slot
    const int box = A.box[ii];
    const int root = A.box_root[box];
    const int self_leaf = A.leaf_of[ii];
    GLane L;
    L.sx = L.sy = L.sz = L.cx = L.cy = L.cz = 0.f;
    L.fx = L.fy = L.fz = 0.f;
    L.ncell = L.nleaf = L.nmac = L.nrecheck = 0;
    L.iters = 0;
    L.fcount = 0;
    const ImgTab* itab = A.img + (size_t)box * A.nimg;
    const int gcentre = (A.ngx * (2 * A.ngy + 1) + A.ngy) * (2 * A.ngz + 1) + A.ngz;
    int gi = -1;               // current image
    int fc = 0, lc = 0, mc = 0;
    const bool any = root >= 0;
    for (;;) {
        const bool last = fc == 0 && gi + 1 >= A.nimg;
        if (lc > kGList - 32 || (fc == 0 && lc > 0)) {
            eval_list<kQuad, kSoft>(A, G.rec, lc, ii, itab[gi], gi == gcentre ? self_leaf : -1, L);
            lc = 0;
        }
        if (mc > kGMix - 32 || (last && mc > 0)) {
            mixed_walks<kQuad, kInside, kSoft, kS>(A, G.mix, mc, itab, ii, self_leaf, gcentre, L);
            mc = 0;
        }
        if (last || !any) break;
        if (fc == 0) {
            // next image: its target points and their bounding box, relative
            // to lane 0's target (hi parts): u = (t_hi - r) + t_lo
            gi++;
            float2 nxy, lxy, nz;
            neg_target(A, ii, itab[gi], nxy, lxy, nz);
            const float rx = __shfl_sync(kFull, -nxy.x, 0);
            const float ry = __shfl_sync(kFull, -nxy.y, 0);
            const float rz = __shfl_sync(kFull, -nz.x, 0);
            const float ux = (-nxy.x - rx) - lxy.x, uy = (-nxy.y - ry) - lxy.y, uz = (-nz.x - rz) - nz.y;
            const float bx0 = warp_min(ux), bx1 = warp_max(ux);
            const float by0 = warp_min(uy), by1 = warp_max(uy);
            const float bz0 = warp_min(uz), bz1 = warp_max(uz);
            __syncwarp();
            if (lane == 0) {
                G.front[0] = root;
                G.box[0] = bx0; G.box[1] = bx1; G.box[2] = by0; G.box[3] = by1;
                G.box[4] = bz0; G.box[5] = bz1;
                G.box[6] = fmaxf(fmaxf(fmaxf(-bx0, bx1), fmaxf(-by0, by1)), fmaxf(-bz0, bz1));
                G.box[7] = rx; G.box[8] = ry; G.box[9] = rz;
            }
            fc = 1;
        }
        __syncwarp();
        const int k = min(32, fc);
        int item = lane < k ? G.front[fc - k + lane] : -1;
        if (item >= A.ecap) {
            // cannot happen for a well-formed tree: record it and drop the cell
            atomicOr(&A.ctl->err, kErrWalk);
            item = -1;
        }
        fc -= k;
        __syncwarp();   // the popped slots are written over below
        // 0 none, 1 accepted cell, 2 open, 3 mixed, 4 leaf
        int cls = 0;
        uint32_t cm = 0;
        float4 ra = make_float4(0.f, 0.f, 0.f, 0.f), rb = ra;
        if (item >= 0) {
            ra = __ldg(&A.ra[item]);
            rb = __ldg(&A.rb[item]);
            const float crit = rb.z;
            if (__float_as_int(crit) < 0) {
                cls = 4;
            } else {
                const float bx0 = G.box[0], bx1 = G.box[1], by0 = G.box[2], by1 = G.box[3];
                const float bz0 = G.box[4], bz1 = G.box[5], ext = G.box[6];
                const float rx = G.box[7], ry = G.box[8], rz = G.box[9];
                // centre of mass relative to the reference point
                const float Dx = (ra.x - rx) + rb.x, Dy = (ra.y - ry) + rb.y, Dz = (ra.z - rz) + ra.w;
                // rounding of D and of the box corners stays below 2^-21
                // (|D| + extent); distances are widened / shortened by it
                const float err = 4.76837158e-7f * (fabsf(Dx) + fabsf(Dy) + fabsf(Dz) + ext);
                const float ax = fmaxf(fmaxf(fmaxf(bx0 - Dx, Dx - bx1), 0.f) - err, 0.f);
                const float ay = fmaxf(fmaxf(fmaxf(by0 - Dy, Dy - by1), 0.f) - err, 0.f);
                const float az = fmaxf(fmaxf(fmaxf(bz0 - Dz, Dz - bz1), 0.f) - err, 0.f);
                const float hx = fmaxf(Dx - bx0, bx1 - Dx) + err;
                const float hy = fmaxf(Dy - by0, by1 - Dy) + err;
                const float hz = fmaxf(Dz - bz0, bz1 - Dz) + err;
                const float rmin2 = fmaf(az, az, fmaf(ay, ay, ax * ax));
                const float rmax2 = fmaf(hz, hz, fmaf(hy, hy, hx * hx));
                if (crit < rmin2 * (1.f - 1e-4f)) {
                    cls = 1;
                    if (kInside) {
                        // the box must also be clear of the cell's cube
                        const float4 ch = __ldg(&A.rc_hi[item]);
                        const float4 cl = __ldg(&A.rc_lo[item]);
                        const float w = ch.w, tol = 1e-5f * w + err;
                        const float cx0 = (ch.x - rx) + cl.x, cy0 = (ch.y - ry) + cl.y,
                                    cz0 = (ch.z - rz) + cl.z;
                        const bool apart = bx1 < cx0 - tol || bx0 > cx0 + w + tol ||
                                           by1 < cy0 - tol || by0 > cy0 + w + tol ||
                                           bz1 < cz0 - tol || bz0 > cz0 + w + tol;
                        if (!apart) cls = 3;
                    }
                } else if (crit > rmax2 * (1.f + 1e-4f)) {
                    cm = __ldg(&A.e_cmask[item]);
                    cls = cm ? 2 : 3;   // a depth-21 group has no child table
                } else {
                    cls = 3;
                }
            }
        }
        // children of opened cells onto the frontier (a cell whose children
        // do not fit is walked as a mixed subtree instead)
        const int nch = cls == 2 ? __popc(cm) : 0;
        int pre = nch;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, pre, o);
            if (lane >= o) pre += t;
        }
        if (cls == 2 && fc + pre > kGFront) cls = 3;
        const unsigned mopen = __ballot_sync(kFull, cls == 2);
        if (cls == 2) {
            int pos = fc + pre - nch;
            const int* ch = A.e_child + 8 * (size_t)item;
            for (uint32_t b = cm; b; b &= b - 1) G.front[pos++] = __ldg(&ch[__ffs(b) - 1]);
        }
        // the pushes are contiguous up to the first cell that did not fit
        const int lastopen = mopen ? 31 - __clz(mopen) : 0;
        const int pushed = mopen ? __shfl_sync(kFull, pre, lastopen) : 0;
        const unsigned macc = __ballot_sync(kFull, cls == 1);
        const unsigned mlist = macc | __ballot_sync(kFull, cls == 4);
        const unsigned mmix = __ballot_sync(kFull, cls == 3);
        const unsigned below = (1u << lane) - 1u;
        if (cls == 1 || cls == 4) {
            // stage the record: the list is evaluated from shared memory
            float4* r = G.rec[lc + __popc(mlist & below)];
            r[0] = ra;
            r[1] = rb;
            if (cls == 1) {
                r[2] = __ldg(&A.rq0[item]);
                r[3] = __ldg(&A.rq1[item]);
            }
        }
        if (cls == 3) G.mix[mc + __popc(mmix & below)] = make_int2(item, gi);
        // opening tests decided for the whole group count for every target:
        // accepted and opened cells (leaves count when evaluated)
        L.ncell += __popc(macc);
        L.nmac += __popc(macc) + __popc(mopen);
        fc += pushed;
        lc += __popc(mlist);
        mc += __popc(mmix);
        L.iters++;
        __syncwarp();
    }
    glane_flush(L);
    if (valid) {
        A.out.ax[i] = A.G * ((double)L.sx - (double)L.cx);
        A.out.ay[i] = A.G * ((double)L.sy - (double)L.cy);
        A.out.az[i] = A.G * ((double)L.sz - (double)L.cz);
        if (A.out.ncell) {
            A.out.ncell[i] = L.ncell;
            A.out.nleaf[i] = L.nleaf;
            A.out.nmac[i] = L.nmac;
        }
    }
    unsigned long long c0 = valid ? L.ncell : 0, c1 = valid ? L.nleaf : 0, c2 = valid ? L.nmac : 0,
                       c3 = valid ? L.nrecheck : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c0 += __shfl_down_sync(kFull, c0, o);
        c1 += __shfl_down_sync(kFull, c1, o);
        c2 += __shfl_down_sync(kFull, c2, o);
        c3 += __shfl_down_sync(kFull, c3, o);
    }
    if (lane == 0) {
        atomicAdd(&A.ctl->n_cell, c0);
        atomicAdd(&A.ctl->n_leaf, c1);
        atomicAdd(&A.ctl->n_mac, c2);
        atomicAdd(&A.ctl->n_recheck, c3);
        atomicAdd(&A.ctl->n_iter, (unsigned long long)L.iters);
    }
}

// Plain FP32 walk with group decisions.  kOne: a single box; otherwise a
// tile whose targets lie in more than one box takes the union walk.
template <bool kQuad, bool kInside, bool kSoft, bool kOne, int kS>
__global__ void __launch_bounds__(kMaxWalkBlock, 4) k_gwalk32(GravArgs A) {
    __shared__ GroupSmem gs[kMaxWalkBlock / 32];
    GroupSmem& G = gs[threadIdx.x >> 5];
    const int n = min(A.ctl->n_live, A.ncap);
    const int ntile = (n + 31) >> 5, q = sm_queue(A.nq);
    for (int t = next_tile(A.tq, A.nq, q, ntile); t >= 0; t = next_tile(A.tq, A.nq, q, ntile)) {
        if (!kOne) {
            const int k = (t << 5) + (threadIdx.x & 31);
            const int b = A.box[tile_slot(A.order, k < n ? k : n - 1)];
            if (!__all_sync(kFull, b == __shfl_sync(kFull, b, 0))) {
                walk32<kQuad, kInside, false, kSoft, false, false, false>(A, nullptr, nullptr, t << 5, n);
                continue;
            }
        }
        walk32g<kQuad, kInside, kSoft, kS>(A, G, t << 5, n);
    }
}

// Learned walk: the network's weights and one queue per warp in shared
// memory; up to 128 registers per thread for the MMA fragments.
template <bool kInside, bool kSoft>
__global__ void __launch_bounds__(kMaxWalkBlock, 2) k_walk32_learn(GravArgs A) {
    __shared__ __align__(16) mlp::Packed w;
    __shared__ __align__(16) LearnQ q[kMaxWalkBlock / 32];
    {
        const uint4* src = reinterpret_cast<const uint4*>(A.wpk);
        uint4* dst = reinterpret_cast<uint4*>(&w);
        for (int k = threadIdx.x; k < (int)(sizeof(mlp::Packed) / 16); k += blockDim.x) dst[k] = src[k];
    }
    __syncthreads();
    const int n = min(A.ctl->n_live, A.ncap);
    const int ntile = (n + 31) >> 5, sq = sm_queue(A.nq);
    for (int t = next_tile(A.tq, A.nq, sq, ntile); t >= 0; t = next_tile(A.tq, A.nq, sq, ntile))
        walk32<true, kInside, false, kSoft, false, true>(A, &q[threadIdx.x >> 5], &w, t << 5, n);
}

// FP64 walk: the same traversal on FP64 records, every opening test in the
// oracle's operation sequence.
template <bool kQuad, bool kInside, bool kPot>
__device__ __forceinline__ void walk64(const GravArgs& A, int wbase, int n) {
    const int lane = threadIdx.x & 31;
    const bool valid = wbase + lane < n;
    const int ii = tile_slot(A.order, valid ? wbase + lane : n - 1);
    const int i = ii;   // the target's slot
    const double px = A.x[ii], py = A.y[ii], pz = A.z[ii];
    const int root = A.box_root[A.box[ii]];
    const int wend = root >= 0 ? A.e_skip[root] : 0;   // end of this box's tree
    const int self_leaf = A.leaf_of[ii];
    const ImgTab* itab = A.img + (size_t)A.box[ii] * A.nimg;
    int gi = 0;
    const double soft2 = A.soft2;
    double ax = 0.0, ay = 0.0, az = 0.0, pot = 0.0;
    int ncell = 0, nleaf = 0, nmac = 0;
    for (int gx = -A.ngx; gx <= A.ngx; gx++)
        for (int gy = -A.ngy; gy <= A.ngy; gy++)
            for (int gz = -A.ngz; gz <= A.ngz; gz++, gi++) {
                const double ox = itab[gi].ox, oy = itab[gi].oy, oz = itab[gi].oz;
                const double tx = __dsub_rn(px, ox), ty = __dsub_rn(py, oy), tz = __dsub_rn(pz, oz);
                const int self = (gx == 0 && gy == 0 && gz == 0) ? self_leaf : -1;
                int next = (valid && root >= 0) ? root : kEnd;
                for (;;) {
                    if (next >= wend) next = kEnd;
                    const int e = (int)__reduce_min_sync(kFull, (unsigned)next);
                    if (e == kEnd) break;
                    const double4_32a a = ld_d4(&A.d_a[e]);
                    const bool act = next == e;
                    if (__double_as_longlong(a.w) < 0) {
                        if (act) {
                            if (e != self) {
                                const double dx = a.x - tx, dy = a.y - ty, dz = a.z - tz;
                                const double r2 = fma(dz, dz, fma(dy, dy, dx * dx)) + soft2;
                                const double inv = rsqrt(r2);
                                const double f = -a.w * (inv * inv * inv);
                                ax = fma(f, dx, ax);
                                ay = fma(f, dy, ay);
                                az = fma(f, dz, az);
                                if (kPot) pot = fma(a.w, inv, pot);
                                nleaf++;
                            }
                            next = e + 1;
                        }
                    } else if (act) {
                        nmac++;
                        bool acc = mac64(a, A.theta2, tx, ty, tz);
                        if (kInside && acc) acc = !inside64(ld_d4(&A.d_c[e]), tx, ty, tz);
                        if (acc) {
                            const double4_32a q0 = ld_d4(&A.d_q0[e]);
                            const double dx = a.x - tx, dy = a.y - ty, dz = a.z - tz;
                            const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
                            const double invs = rsqrt(r2 + soft2);
                            const double f = q0.x * (invs * invs * invs);
                            ax = fma(f, dx, ax);
                            ay = fma(f, dy, ay);
                            az = fma(f, dz, az);
                            if (kPot) pot = fma(-q0.x, invs, pot);
                            if (kQuad) {
                                const double4_32a q1 = ld_d4(&A.d_q1[e]);
                                const double inv = rsqrt(r2);
                                const double inv2 = inv * inv;
                                const double qx = fma(q1.y, dz, fma(q1.x, dy, q0.y * dx));
                                const double qy = fma(q1.z, dz, fma(q0.z, dy, q1.x * dx));
                                const double qz = fma(q0.w, dz, fma(q1.z, dy, q1.y * dx));
                                const double dqd = fma(dz, qz, fma(dy, qy, dx * qx));
                                const double inv5 = inv2 * inv2 * inv;
                                const double c = 2.5 * dqd * (inv5 * inv2);
                                ax = fma(c, dx, fma(-inv5, qx, ax));
                                ay = fma(c, dy, fma(-inv5, qy, ay));
                                az = fma(c, dz, fma(-inv5, qz, az));
                                if (kPot) pot = fma(-0.5 * dqd, inv5, pot);
                            }
                            ncell++;
                            next = A.e_skip[e];
                        } else {
                            next = e + 1;
                        }
                    }
                }
            }
    if (valid) {
        A.out.ax[i] = A.G * ax;
        A.out.ay[i] = A.G * ay;
        A.out.az[i] = A.G * az;
        if (kPot) A.out.phi[i] = A.G * pot;
        if (A.out.ncell) {
            A.out.ncell[i] = ncell;
            A.out.nleaf[i] = nleaf;
            A.out.nmac[i] = nmac;
        }
    }
    unsigned long long c0 = valid ? ncell : 0, c1 = valid ? nleaf : 0, c2 = valid ? nmac : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c0 += __shfl_down_sync(kFull, c0, o);
        c1 += __shfl_down_sync(kFull, c1, o);
        c2 += __shfl_down_sync(kFull, c2, o);
    }
    if (lane == 0) {
        atomicAdd(&A.ctl->n_cell, c0);
        atomicAdd(&A.ctl->n_leaf, c1);
        atomicAdd(&A.ctl->n_mac, c2);
    }
}

template <bool kQuad, bool kInside, bool kPot>
__global__ void __launch_bounds__(kMaxWalkBlock) k_walk64(GravArgs A) {
    const int n = min(A.ctl->n_live, A.ncap);
    const int ntile = (n + 31) >> 5, q = sm_queue(A.nq);
    for (int t = next_tile(A.tq, A.nq, q, ntile); t >= 0; t = next_tile(A.tq, A.nq, q, ntile))
        walk64<kQuad, kInside, kPot>(A, t << 5, n);
}

struct CollArgs {
    const double *x, *y, *z, *r;
    const int32_t *id, *box;
    Rec4 ra, rb;
    const int32_t *box_root, *e_skip;
    const BoxP* boxes;
    Ctl* ctl;
    uint64_t* pair_key;
    int pair_cap;
    int ncap;
    int ngx, ngy, ngz;
    int half_step_offset;
    double t0, half_dt;
    const ImgTab* img;   // [box][image] offsets at the time of this search
    int nimg;
    int32_t* tq;         // tile queues (emptied by the image-table launch)
    int nq;
    float rmaxf;         // largest radius, rounded up (box records)
    const int32_t* e_top;   // sphere records: largest particle slot below each cell
    const uint32_t* order;  // tile order of the targets (nullptr: Morton order of the slots)
};

// Overlap test of Sect. 5.1 on the canonical orientation (a = lower id, b
// seen through image offset o), operation for operation as the oracle.
// kNeg: the offset is -o (b + (-o) and b - o round identically in IEEE
// arithmetic, so no negated copy of o is formed).
template <bool kNeg = false>
__device__ __forceinline__ bool overlap64(double xa, double ya, double za, double ra, double xb,
                                          double yb, double zb, double rb, double ox, double oy,
                                          double oz) {
    const double rx = __dsub_rn(kNeg ? __dsub_rn(xb, ox) : __dadd_rn(xb, ox), xa);
    const double ry = __dsub_rn(kNeg ? __dsub_rn(yb, oy) : __dadd_rn(yb, oy), ya);
    const double rz = __dsub_rn(kNeg ? __dsub_rn(zb, oz) : __dadd_rn(zb, oz), za);
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(rx, rx), __dmul_rn(ry, ry)), __dmul_rn(rz, rz));
    const double sr = __dadd_rn(ra, rb);
    return r2 < __dmul_rn(sr, sr);
}

// Tree collision search (Sect. 5.2): descend while the distance from the
// target point to a cell's centre is below R_i + R_max + (sqrt(3)/2) w (Eq. 3,
// tested in FP32 with a 2e-5 relative margin so that no overlap is pruned);
// kAABB: while the distance to the box of the cell's particles is below
// R_i + R_max (records of build_collision_aabb; a subset of Eq. 3's volume
// that still holds every overlap).
// Each unordered pair is examined once, from its lower slot (the other
// particle reaches it through the opposite image), so a subtree whose
// particles all sit at slots <= i is skipped as well.  A leaf's overlap is
// decided in FP32 on hi/lo positions (distance good to ~1e-7 relative) unless
// d^2 lies within 1e-4 of (R_a + R_b)^2; only those pairs get the exact FP64
// test in the oracle's operation order on the canonical orientation (lower
// id a, image of b as seen from a).  On GB300 an FP64 instruction occupies
// the SM's FP64 pipe 16 cycles per warp, so the exact test on every overlap
// kept that pipe busy for most of the search.
// kCount: also count the entries the targets test (nodes visited) and the
// warp iterations; a separate variant, since the counters cost the
// 32-register search about 9% of its time in spilled registers.
template <bool kAABB, bool kCount>
__device__ __forceinline__ void collide(const CollArgs& A, int wbase, int n) {
    const int lane = threadIdx.x & 31;
    const bool valid = wbase + lane < n;
    const int ii = tile_slot(A.order, valid ? wbase + lane : n - 1);
    const int i = ii;   // the target's slot
    const double px = A.x[ii], py = A.y[ii], pz = A.z[ii], pr = A.r[ii];
    const int pid = A.id[ii];
    const int root = A.box_root[A.box[ii]];
    const int wend = root >= 0 ? A.e_skip[root] : 0;   // end of this box's tree
    const float prf = (float)pr;
    float phx, plx, phy, ply, phz, plz;
    split_d(px, phx, plx);
    split_d(py, phy, ply);
    split_d(pz, phz, plz);
    const ImgTab* itab = A.img + (size_t)A.box[ii] * A.nimg;
    int gi = 0;
    // kCount: entries the warp's targets tested and warp iterations
    // (both warp-uniform)
    unsigned nvis = 0, siter = 0;
    for (int gx = -A.ngx; gx <= A.ngx; gx++)
        for (int gy = -A.ngy; gy <= A.ngy; gy++)
            for (int gz = -A.ngz; gz <= A.ngz; gz++, gi++) {
                const int code = (gx + 7) | ((gy + 7) << 4) | ((gz + 7) << 8);
                float thx, thy, thz, tlx, tly, tlz;
                {
                    const float4 oh = itab[gi].hi, ol = itab[gi].lo;
                    sub_hilo(phx, plx, oh.x, ol.x, thx, tlx);
                    sub_hilo(phy, ply, oh.y, ol.y, thy, tly);
                    sub_hilo(phz, plz, oh.z, ol.z, thz, tlz);
                }
                const float2 nth = make_float2(-thx, -thy), ntl = make_float2(-tlx, -tly);
                int next = (valid && root >= 0) ? root : kEnd;
                for (;;) {
                    if (next >= wend) next = kEnd;
                    const int e = (int)__reduce_min_sync(kFull, (unsigned)next);
                    if (e == kEnd) break;
                    const float4 ra = __ldg(&A.ra[e]);
                    const bool act = next == e;
                    if (kCount) {
                        nvis += __popc(__ballot_sync(kFull, act));
                        siter++;
                    }
                    bool hit = false;
                    uint64_t key = 0;
                    if (__float_as_int(ra.w) < 0) {
                        if (act) {
                            const int j = ~__float_as_int(ra.w);
                            if (j > i) {
                                const float4 rb = __ldg(&A.rb[e]);
                                const float2 dxy = __fadd2_rn(__fadd2_rn(make_float2(ra.x, ra.y), nth),
                                                              __fadd2_rn(make_float2(rb.x, rb.y), ntl));
                                const float dx = dxy.x, dy = dxy.y;
                                const float dz = (ra.z - thz) + (rb.z - tlz);
                                const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                                const float sr = prf + rb.w;
                                const float s2 = sr * sr;
                                if (d2 < s2 * 1.0001f) {
                                    const int jid = A.id[j];
                                    const bool low = pid < jid;
                                    if (d2 < s2 * 0.9999f) {
                                        // clear of the threshold (the FP32 distance is good to
                                        // ~1e-7): an overlap without FP64 work
                                        hit = true;
                                    } else {
                                        const double ox = itab[gi].ox, oy = itab[gi].oy, oz = itab[gi].oz;
                                        // j the lower id: this particle is its image -g, whose
                                        // offset is exactly -o (the table is symmetric)
                                        hit = low ? overlap64(px, py, pz, pr, A.x[j], A.y[j], A.z[j],
                                                              A.r[j], ox, oy, oz)
                                                  : overlap64<true>(A.x[j], A.y[j], A.z[j], A.r[j], px,
                                                                    py, pz, pr, ox, oy, oz);
                                    }
                                    const int ncode = (-gx + 7) | ((-gy + 7) << 4) | ((-gz + 7) << 8);
                                    key = low ? ((uint64_t)pid << 36) | ((uint64_t)jid << 12) | (uint64_t)code
                                              : ((uint64_t)jid << 36) | ((uint64_t)pid << 12) | (uint64_t)ncode;
                                }
                            }
                            next = e + 1;
                        }
                    } else if (act) {
                        const float4 rb = __ldg(&A.rb[e]);
                        if (kAABB) {
                            // distance to the cell's box [ra.xyz, rb.xyz] of particle
                            // positions; opened unless farther than R_i + R_max, or
                            // unless every particle below sits at a slot <= i (those
                            // pairs are examined from the other particle)
                            // (t - b) + l = -((b - t) - l) exactly, so the upper side
                            // comes negated out of the same packed adds
                            const float2 u = __fadd2_rn(__fadd2_rn(make_float2(ra.x, ra.y), nth), ntl);
                            const float2 v = __fadd2_rn(__fadd2_rn(make_float2(rb.x, rb.y), nth), ntl);
                            const float ex = fmaxf(fmaxf(u.x, -v.x), 0.f);
                            const float ey = fmaxf(fmaxf(u.y, -v.y), 0.f);
                            const float ez = fmaxf(fmaxf((ra.z - thz) - tlz, (thz - rb.z) + tlz), 0.f);
                            const float d2 = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
                            const float lim = (prf + A.rmaxf) * 1.0001f +
                                              4e-7f * (fabsf(thx) + fabsf(thy) + fabsf(thz));
                            next = (__float_as_int(ra.w) > i && d2 < lim * lim) ? e + 1
                                                                                : __float_as_int(rb.w);
                        } else {
                            const float2 dxy = __fadd2_rn(__fadd2_rn(make_float2(ra.x, ra.y), nth),
                                                          __fadd2_rn(make_float2(rb.x, rb.y), ntl));
                            const float dx = dxy.x, dy = dxy.y;
                            const float dz = (ra.z - thz) + (rb.z - tlz);
                            const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                            const float lim = (prf + ra.w) * 1.00002f;
                            next = (__ldg(&A.e_top[e]) > i && d2 < lim * lim) ? e + 1
                                                                              : __float_as_int(rb.w);
                        }
                    }
                    const unsigned hits = __ballot_sync(kFull, hit);
                    if (hits) {
                        int base = 0;
                        const int leader = __ffs(hits) - 1;
                        if (lane == leader) base = atomicAdd(&A.ctl->pair_count, __popc(hits));
                        base = __shfl_sync(kFull, base, leader);
                        if (hit) {
                            const int slot = base + __popc(hits & ((1u << lane) - 1u));
                            if (slot < A.pair_cap) A.pair_key[slot] = key;
                            else atomicOr(&A.ctl->err, kErrPairOverflow);
                        }
                    }
                }
            }
    if (kCount && lane == 0) {
        atomicAdd(&A.ctl->n_visit, (unsigned long long)nvis);
        atomicAdd(&A.ctl->n_siter, (unsigned long long)siter);
    }
}

// At most 32 registers (8 blocks of 256 threads per SM, every warp slot
// resident): the search is latency-bound, and going from 40 resident warps
// per SM (48 registers) to 48 (40) and 64 (32, with a few spilled values)
// took 4% and another 2% off it.
template <bool kAABB, bool kCount = false>
__global__ void __launch_bounds__(kMaxWalkBlock, 8) k_collide(CollArgs A) {
    const int n = min(A.ctl->n_live, A.ncap);
    const int ntile = (n + 31) >> 5, q = sm_queue(A.nq);
    for (int t = next_tile(A.tq, A.nq, q, ntile); t >= 0; t = next_tile(A.tq, A.nq, q, ntile))
        collide<kAABB, kCount>(A, t << 5, n);
}

}  // namespace

int build_image_table(const BoxP* boxes, const Ctl* ctl, const SimC& C, int half_step_offset, ImgTab* tab,
                      cudaStream_t s, int32_t* tq, int nq) {
    const int nimg = (2 * C.ngx + 1) * (2 * C.ngy + 1) * (2 * C.ngz + 1);
    const int nqw = tq ? nq * kTileQStride : 0;
    const int nt = max((C.nbox + 1) * nimg, nqw);
    k_img_table<<<ceil_div(nt, 128), 128, 0, s>>>(boxes, ctl, C.t0, C.half_dt, half_step_offset, C.nbox,
                                                   C.ngx, C.ngy, C.ngz, tab, tq, nqw);
    return nimg;
}

namespace {

// Resident blocks per SM of each walk / search kernel at each block size,
// queried once: a stream capture must not see the first query of a kernel.
struct Residency {
    const void* fn;
    int block, per_sm;
};
std::mutex g_res_mu;
std::vector<Residency> g_res;
int g_nsm = 0;

int query_residency(const void* fn, int block) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, 0) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
    }
    return max(per_sm, 1);
}

int residency(const void* fn, int block) {
    std::lock_guard<std::mutex> lk(g_res_mu);
    for (const Residency& r : g_res)
        if (r.fn == fn && r.block == block) return r.per_sm;
    const int per_sm = query_residency(fn, block);
    g_res.push_back({fn, block, per_sm});
    return per_sm;
}

// Persistent grid of kernel fn: the blocks that fit on the GPU at once, but
// no more than the blocks that one target per thread would need.
template <typename F>
int persistent_grid(F fn, int block, int cap_n) {
    const int need = ceil_div(cap_n, block);
    const int fit = max(g_nsm, 1) * residency(reinterpret_cast<const void*>(fn), block);
    return max(1, min(need, fit));
}

template <typename F>
void prepare_one(F fn) {
    for (int b : {64, 128, 256}) residency(reinterpret_cast<const void*>(fn), b);
}

}  // namespace

int walk_prepare() {
    {
        std::lock_guard<std::mutex> lk(g_res_mu);
        if (g_nsm > 0) return g_nsm;
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        g_nsm = nsm;
    }
    prepare_one(k_walk32<true, true, false, true>); prepare_one(k_walk32<true, true, false, false>);
    prepare_one(k_walk32<true, false, false, true>); prepare_one(k_walk32<true, false, false, false>);
    prepare_one(k_walk32<false, true, false, true>); prepare_one(k_walk32<false, true, false, false>);
    prepare_one(k_walk32<false, false, false, true>); prepare_one(k_walk32<false, false, false, false>);
    prepare_one(k_walk32<true, true, false, true, false, true>);
    prepare_one(k_walk32<true, true, false, false, false, true>);
    prepare_one(k_walk32<true, false, false, true, false, true>);
    prepare_one(k_walk32<true, false, false, false, false, true>);
    prepare_one(k_walk32<false, true, false, true, false, true>);
    prepare_one(k_walk32<false, true, false, false, false, true>);
    prepare_one(k_walk32<false, false, false, true, false, true>);
    prepare_one(k_walk32<false, false, false, false, false, true>);
    prepare_one(k_walk32<true, true, false, true, true>); prepare_one(k_walk32<true, true, false, false, true>);
    prepare_one(k_walk32<true, false, false, true, true>); prepare_one(k_walk32<true, false, false, false, true>);
    prepare_one(k_walk32_learn<true, true>); prepare_one(k_walk32_learn<true, false>);
    prepare_one(k_walk32_learn<false, true>); prepare_one(k_walk32_learn<false, false>);
    prepare_one(k_walk64<true, true, true>); prepare_one(k_walk64<true, true, false>);
    prepare_one(k_walk64<true, false, true>); prepare_one(k_walk64<true, false, false>);
    prepare_one(k_walk64<false, true, true>); prepare_one(k_walk64<false, true, false>);
    prepare_one(k_walk64<false, false, true>); prepare_one(k_walk64<false, false, false>);
#define RB_PREP_G(Q, I, S) \
    prepare_one(k_gwalk32<Q, I, S, true, 4>); prepare_one(k_gwalk32<Q, I, S, false, 4>)
    RB_PREP_G(true, true, true); RB_PREP_G(true, true, false);
    RB_PREP_G(true, false, true); RB_PREP_G(true, false, false);
    RB_PREP_G(false, true, true); RB_PREP_G(false, true, false);
    RB_PREP_G(false, false, true); RB_PREP_G(false, false, false);
#undef RB_PREP_G
    prepare_one(k_collide<true>);
    prepare_one(k_collide<false>);
    prepare_one(k_collide<true, true>);
    prepare_one(k_collide<false, true>);
    return g_nsm;
}

void gravity_walk(const Tree& T, const PSet& P, Ctl* ctl, const BoxP* boxes, const SimC& C,
                  int walk_mode, int half_step_offset, const WalkOut& out, bool potential,
                  bool counts, cudaStream_t s, const WalkRecord* rec, int block,
                  const WalkLearn* learn, int group) {
    block = (block == 64 || block == 256) ? block : 128;
    group = group == 4 ? 4 : 0;
    if (T.cap_n <= 0) return;
    GravArgs A;
    A.ecap = T.cap_e;
    A.e_count = T.e_count;
    A.wpk = learn ? learn->w : nullptr;
    A.req = nullptr; A.req_count = nullptr; A.req_cap = 0;
    A.band_scale = 0.f; A.thresh = 0u; A.seed = 0u;
    if (rec) {
        A.req = rec->req; A.req_count = rec->count; A.req_cap = rec->cap;
        A.band_scale = rec->band_scale; A.thresh = rec->thresh; A.seed = rec->seed;
    }
    A.x = P.x; A.y = P.y; A.z = P.z; A.box = P.box;
    A.ra = T.ra; A.rb = T.rb; A.rq0 = T.rq0; A.rq1 = T.rq1; A.rc_hi = T.rc_hi; A.rc_lo = T.rc_lo;
    A.d_a = reinterpret_cast<const double4_32a*>(T.d_a);
    A.d_q0 = reinterpret_cast<const double4_32a*>(T.d_q0);
    A.d_q1 = reinterpret_cast<const double4_32a*>(T.d_q1);
    A.d_c = reinterpret_cast<const double4_32a*>(T.d_c);
    A.e_skip = T.e_skip; A.leaf_of = T.leaf_of; A.box_root = T.box_root;
    A.e_child = T.e_child; A.e_cmask = T.e_cmask;
    A.order = T.order;
    A.boxes = boxes; A.ctl = ctl;
    A.out = out;
    if (!counts) { A.out.ncell = nullptr; A.out.nleaf = nullptr; A.out.nmac = nullptr; }
    A.ncap = T.cap_n;
    A.ngx = C.ngx; A.ngy = C.ngy; A.ngz = C.ngz;
    A.half_step_offset = half_step_offset;
    A.G = C.G; A.theta2 = C.theta2; A.soft2 = C.soft2; A.t0 = C.t0; A.half_dt = C.half_dt;
    A.soft2f = (float)C.soft2;
    const bool inside = C.theta2 > (1.0 / 3.0);
    const bool quad = C.quadrupole != 0;
    const bool soft = C.soft2 > 0.0;
    A.img = T.img;
    A.tq = T.tq;
    A.nq = T.nq;
    A.nimg = build_image_table(boxes, ctl, C, half_step_offset, T.img, s, T.tq, T.nq);
    // every kernel below runs the persistent grid that fits on the GPU
#define RB_LAUNCH(...) __VA_ARGS__<<<persistent_grid(__VA_ARGS__, block, T.cap_n), block, 0, s>>>(A)
#define RB_W32G(Q, I, S, ONE) RB_LAUNCH(k_gwalk32<Q, I, S, ONE, 4>)
#define RB_W32(Q, I, PO, S)                                                \
    do {                                                                   \
        if (group == 0) {                                                  \
            if (C.nbox == 1) RB_LAUNCH(k_walk32<Q, I, PO, S, false, true>); \
            else RB_LAUNCH(k_walk32<Q, I, PO, S>);                          \
        } else if (C.nbox == 1) {                                          \
            RB_W32G(Q, I, S, true);                                        \
        } else {                                                           \
            RB_W32G(Q, I, S, false);                                       \
        }                                                                  \
    } while (0)
#define RB_W64(Q, I, PO) RB_LAUNCH(k_walk64<Q, I, PO>)
    if (learn && !potential) {
        // FP32 walk with the learned correction of band cells (quadrupole on)
        A.band_scale = learn->band_scale;
        if (inside) {
            if (soft) RB_LAUNCH(k_walk32_learn<true, true>);
            else RB_LAUNCH(k_walk32_learn<true, false>);
        } else {
            if (soft) RB_LAUNCH(k_walk32_learn<false, true>);
            else RB_LAUNCH(k_walk32_learn<false, false>);
        }
    } else if (rec) {
        // FP32 walk that also records accepted band cells (quadrupole on)
        if (inside) {
            if (soft) RB_LAUNCH(k_walk32<true, true, false, true, true>);
            else RB_LAUNCH(k_walk32<true, true, false, false, true>);
        } else {
            if (soft) RB_LAUNCH(k_walk32<true, false, false, true, true>);
            else RB_LAUNCH(k_walk32<true, false, false, false, true>);
        }
    } else if (walk_mode == 0 || potential) {
        if (quad) {
            if (inside) { if (potential) RB_W64(true, true, true); else RB_W64(true, true, false); }
            else { if (potential) RB_W64(true, false, true); else RB_W64(true, false, false); }
        } else {
            if (inside) { if (potential) RB_W64(false, true, true); else RB_W64(false, true, false); }
            else { if (potential) RB_W64(false, false, true); else RB_W64(false, false, false); }
        }
    } else {
        if (quad) {
            if (inside) { if (soft) RB_W32(true, true, false, true); else RB_W32(true, true, false, false); }
            else { if (soft) RB_W32(true, false, false, true); else RB_W32(true, false, false, false); }
        } else {
            if (inside) { if (soft) RB_W32(false, true, false, true); else RB_W32(false, true, false, false); }
            else { if (soft) RB_W32(false, false, false, true); else RB_W32(false, false, false, false); }
        }
    }
#undef RB_W32
#undef RB_W32G
#undef RB_W64
}

void collision_search(const Tree& T, const PSet& P, Ctl* ctl, const BoxP* boxes, const SimC& C,
                      const Pairs& PR, int half_step_offset, cudaStream_t s, int block, bool aabb,
                      double rmax, bool count) {
    if (T.cap_n <= 0) return;
    block = (block == 64 || block == 256) ? block : 128;
    CollArgs A;
    A.rmaxf = (float)rmax;
    if ((double)A.rmaxf < rmax) A.rmaxf = nextafterf(A.rmaxf, FLT_MAX);
    A.x = P.x; A.y = P.y; A.z = P.z; A.r = P.r; A.id = P.id; A.box = P.box;
    A.ra = T.ra; A.rb = T.rb; A.box_root = T.box_root; A.e_skip = T.e_skip; A.boxes = boxes;
    A.e_top = T.e_top;
    A.order = T.order;
    A.ctl = ctl;
    A.pair_key = PR.key; A.pair_cap = PR.cap; A.ncap = T.cap_n;
    A.ngx = C.ngx; A.ngy = C.ngy; A.ngz = C.ngz;
    A.half_step_offset = half_step_offset; A.t0 = C.t0; A.half_dt = C.half_dt;
    A.img = T.img;
    A.tq = T.tq;
    A.nq = T.nq;
    A.nimg = build_image_table(boxes, ctl, C, half_step_offset, T.img, s, T.tq, T.nq);
    if (count) {
        if (aabb) RB_LAUNCH(k_collide<true, true>);
        else RB_LAUNCH(k_collide<false, true>);
    } else if (aabb) {
        RB_LAUNCH(k_collide<true>);
    } else {
        RB_LAUNCH(k_collide<false>);
    }
#undef RB_LAUNCH
}

}  // namespace rb
