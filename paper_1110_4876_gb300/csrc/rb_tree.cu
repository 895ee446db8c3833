// rb_tree.cu -- the octree of Sect. 4.2 built from Morton-sorted particles,
// its cell moments and the records the walks read.
//
// Cells are the key prefixes (3 bits per depth) shared by two or more
// particles that split at the next depth (or sit at the depth cap of 21,
// where they are leaf groups).  Cells with a single occupied octant are
// skipped: they hold the same particles, centre of mass and quadrupole as
// that octant and a wider cell is never accepted where the narrower one is
// not, so the forces equal those of the paper's insertion tree.
//
// Between sorted particles i and i+1 ("split" i) the shared prefix depth is
// delta_i.  A cell of depth v is a maximal run of splits with delta >= v that
// contains a split with delta == v; its first such split is its
// representative.  Range minima of delta come straight from the keys
// (clz of the xor of the run's end keys), so each split finds its run with a
// galloping search.  Cells are laid out in depth-first pre-order together
// with one leaf entry per particle: entry order is (first particle, depth),
// and a per-particle bitmask of the depths of cells starting there gives
// every entry's position after one scan.
#include <algorithm>
#include <cfloat>

#include "rb_internal.cuh"

namespace rb {
namespace {

template <bool kMultiBox>
__device__ __forceinline__ int lcp_level(const uint64_t* __restrict__ key,
                                         const int32_t* __restrict__ box, int a, int b) {
    if (kMultiBox && box[a] != box[b]) return -1;
    const uint64_t x = key[a] ^ key[b];
    if (x == 0ull) return kMaxDepth;
    return (__clzll((long long)x) - 1) / 3;
}

// One thread per split i in [0, n - 2]: find the run of cell depth
// v = delta_i; if i represents its cell, record the particle range and mark
// the cell's depth in mask[first].
template <bool kMultiBox>
__global__ void __launch_bounds__(256) k_nodes(const uint64_t* __restrict__ key,
                                               const int32_t* __restrict__ box,
                                               const Ctl* __restrict__ ctl, int ncap,
                                               int32_t* __restrict__ node_a,
                                               int32_t* __restrict__ node_b,
                                               int8_t* __restrict__ node_v,
                                               uint32_t* __restrict__ mask) {
    const int n = min(ctl->n_live, ncap);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const int v = lcp_level<kMultiBox>(key, box, i, i + 1);
    int8_t outv = -1;
    if (v >= 0) {
        // leftmost particle a with min(delta_a .. delta_i) >= v
        int good = i, step = 1, bad = -1;
        for (;;) {
            const int c = i - step;
            if (c < 0) { bad = -1; break; }
            if (lcp_level<kMultiBox>(key, box, c, i + 1) < v) { bad = c; break; }
            good = c;
            step <<= 1;
        }
        while (good - bad > 1) {
            const int mid = (good + bad) >> 1;
            if (lcp_level<kMultiBox>(key, box, mid, i + 1) >= v) good = mid; else bad = mid;
        }
        const int a = good;
        const bool rep = (a == i) || (lcp_level<kMultiBox>(key, box, a, i) > v);
        node_a[i] = a;
        outv = (int8_t)(v + 32);   // the split's cell; its representative is another split
        if (rep) {
            // rightmost particle b with min(delta_i .. delta_{b-1}) >= v
            int g2 = i + 1, st = 1, b2 = n;
            for (;;) {
                const int c = i + 1 + st;
                if (c >= n) { b2 = n; break; }
                if (lcp_level<kMultiBox>(key, box, i, c) < v) { b2 = c; break; }
                g2 = c;
                st <<= 1;
            }
            while (b2 - g2 > 1) {
                const int mid = (g2 + b2) >> 1;
                if (lcp_level<kMultiBox>(key, box, i, mid) >= v) g2 = mid; else b2 = mid;
            }
            node_b[i] = g2;
            outv = (int8_t)v;
            atomicOr(&mask[a], 1u << v);
        }
    }
    node_v[i] = outv;
}

__global__ void __launch_bounds__(256) k_entry_counts(const uint32_t* __restrict__ mask,
                                                      const Ctl* __restrict__ ctl, int ncap,
                                                      int32_t* __restrict__ start) {
    const int n = min(ctl->n_live, ncap);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) start[i] = 1 + __popc(mask[i]);
}

// Entries in pre-order: cells (from their representative split) and leaves.
__global__ void __launch_bounds__(256) k_emit(const uint32_t* __restrict__ mask,
                                              const int32_t* __restrict__ start,
                                              const int32_t* __restrict__ node_a,
                                              const int32_t* __restrict__ node_b,
                                              const int8_t* __restrict__ node_v,
                                              const Ctl* __restrict__ ctl, int ncap,
                                              int32_t* __restrict__ e_first,
                                              int32_t* __restrict__ e_count,
                                              int32_t* __restrict__ e_skip,
                                              int8_t* __restrict__ e_level,
                                              int32_t* __restrict__ leaf_of,
                                              const uint64_t* __restrict__ key,
                                              int32_t* __restrict__ e_child,
                                              uint32_t* __restrict__ e_cmask) {
    const int n = min(ctl->n_live, ncap);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t mk = mask[i];
    const int li = start[i] + __popc(mk);
    e_first[li] = i;
    e_count[li] = 1;
    e_skip[li] = li + 1;
    e_level[li] = 22;
    leaf_of[i] = li;
    if (i < n - 1) {
        const int vv = node_v[i];
        if (vv >= 0) {
            const int v = vv & 31;
            const int a = node_a[i];
            const int idx = start[a] + __popc(mask[a] & ((1u << v) - 1u));   // the split's cell
            if (vv < 32) {
                const int b = node_b[i];
                e_first[idx] = a;
                e_count[idx] = b - a + 1;
                e_skip[idx] = start[b + 1];
                e_level[idx] = (int8_t)v;
            }
            // child table (not for depth-21 groups, whose members share one key):
            // particles i and i + 1 part at depth v + 1, so the child of cell idx
            // that starts at particle i + 1 is its shallowest entry there; the
            // representative also enters the first child, entry idx + 1
            if (v < kMaxDepth) {
                const int sh = 3 * (kMaxDepth - 1 - v);
                const int o = (int)((key[i + 1] >> sh) & 7ull);
                e_child[8 * (size_t)idx + o] = start[i + 1];
                atomicOr(&e_cmask[idx], 1u << o);
                if (vv < 32) {
                    const int o0 = (int)((key[a] >> sh) & 7ull);
                    e_child[8 * (size_t)idx + o0] = idx + 1;
                    atomicOr(&e_cmask[idx], 1u << o0);
                }
            }
        }
    }
}

// Box ranges in sorted order (empty boxes get empty ranges) and box roots.
__global__ void __launch_bounds__(256) k_box_ranges(const int32_t* __restrict__ box,
                                                    const Ctl* __restrict__ ctl, int ncap, int nbox,
                                                    int32_t* __restrict__ box_first) {
    const int n = min(ctl->n_live, ncap);
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (n == 0) {
        if (p <= nbox) box_first[p] = 0;
        return;
    }
    if (p >= n) return;
    const int b = box[p];
    const int prev = p == 0 ? -1 : box[p - 1];
    for (int q = prev + 1; q <= b; q++) box_first[q] = p;
    if (p == n - 1)
        for (int q = b + 1; q <= nbox; q++) box_first[q] = n;
}

// Root entry of each box's tree, -1 for an empty box; entry nbox, -1, is the
// root of the box that particles removed by an open boundary carry (nbox):
// those still hold slots of the gravity tree when the step's collision
// search runs on it, and search nothing.
__global__ void k_box_roots(const int32_t* __restrict__ box_first,
                            const int32_t* __restrict__ start, int nbox,
                            int32_t* __restrict__ box_root) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > nbox) return;
    box_root[b] = b < nbox && box_first[b] < box_first[b + 1] ? start[box_first[b]] : -1;
}


__device__ __forceinline__ uint32_t compact3(uint64_t x) {
    x &= 0x1249249249249249ull;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
    x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
    x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
    x = (x ^ (x >> 32)) & 0x1fffffull;
    return (uint32_t)x;
}

__device__ __forceinline__ void split_hilo(double v, float& hi, float& lo) {
    hi = __double2float_rn(v);
    lo = __double2float_rn(v - (double)hi);
}

// Integer cell index of depth v along each axis, from a member's key.
__device__ __forceinline__ void cell_index(uint64_t key, int v, double& ix, double& iy, double& iz) {
    const int sh = kMaxDepth - v;
    ix = (double)(compact3(key >> 2) >> sh);
    iy = (double)(compact3(key >> 1) >> sh);
    iz = (double)(compact3(key) >> sh);
}

struct GravRecArgs {
    const double *x, *y, *z, *m;
    const int32_t *box, *id;
    bool has_test;   // some particles are test particles (source mass 0)
    const uint64_t* key;
    const BoxP* boxes;
    const int32_t *e_first, *e_skip, *e_child, *leaf_of;
    const uint32_t* e_cmask;
    const int8_t* e_level;
    int32_t* e_arrive;
    double4_32a *d_a, *d_q0, *d_q1, *d_c;
    Rec4 ra, rb, rq0, rq1, rc_hi, rc_lo;
    const Ctl* ctl;
    int ncap;
    double crit_scale;  // 1 / theta^2
    bool fp32, inside;
};

// Leaf records (FP64 and FP32) of every particle.
__global__ void __launch_bounds__(256) k_leaf_records(GravRecArgs A) {
    const int n = min(A.ctl->n_live, A.ncap);
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int e = A.leaf_of[p];
    const double x = A.x[p], y = A.y[p], z = A.z[p];
    const double m = A.has_test ? source_mass(A.boxes[A.box[p]], A.id[p], A.m[p]) : A.m[p];
    A.d_a[e] = make_double4_32a(x, y, z, -m);
    if (A.fp32) {
        float hx, lx, hy, ly, hz, lz;
        split_hilo(x, hx, lx);
        split_hilo(y, hy, ly);
        split_hilo(z, hz, lz);
        A.ra[e] = make_float4(hx, hy, hz, lz);
        A.rb[e] = make_float4(lx, ly, -(float)m, __int_as_float(e + 1));
    }
}

// Cells per depth: counts (block histograms, one atomic per depth and
// block), offsets, then the lists.  lvl[0..22]: counts, lvl[32..54]: offsets,
// lvl[64..86]: fill cursors.
__global__ void __launch_bounds__(256) k_level_count(const int8_t* __restrict__ e_level,
                                                     const Ctl* __restrict__ ctl, int ecap,
                                                     int32_t* __restrict__ lvl) {
    __shared__ int h[23];
    if (threadIdx.x < 23) h[threadIdx.x] = 0;
    __syncthreads();
    const int E = min(ctl->n_entries, ecap);
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < E) {
        const int v = e_level[k];
        if (v < 22) atomicAdd(&h[v], 1);
    }
    __syncthreads();
    if (threadIdx.x < 22 && h[threadIdx.x]) atomicAdd(&lvl[threadIdx.x], h[threadIdx.x]);
}

__global__ void k_level_offsets(int32_t* lvl) {
    int s = 0;
    for (int d = 0; d < 22; d++) {
        lvl[32 + d] = s;
        lvl[64 + d] = s;
        s += lvl[d];
    }
}

__global__ void __launch_bounds__(256) k_level_fill(const int8_t* __restrict__ e_level,
                                                    const Ctl* __restrict__ ctl, int ecap,
                                                    int32_t* __restrict__ lvl,
                                                    int32_t* __restrict__ list) {
    __shared__ int h[23], base[23];
    if (threadIdx.x < 23) h[threadIdx.x] = 0;
    __syncthreads();
    const int E = min(ctl->n_entries, ecap);
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    int v = 22, mine = 0;
    if (k < E) {
        v = e_level[k];
        if (v < 22) mine = atomicAdd(&h[v], 1);
    }
    __syncthreads();
    if (threadIdx.x < 22 && h[threadIdx.x]) base[threadIdx.x] = atomicAdd(&lvl[64 + threadIdx.x], h[threadIdx.x]);
    __syncthreads();
    if (v < 22) list[base[v] + mine] = k;
}

// The cells of one depth.  A cell's moments come from its children (deeper
// cells, done by earlier launches, or particle leaves) in one pass: about the
// first child's position o, M = sum M_c, S = sum M_c d_c and
// Q_o = sum [Q_c + M_c (3 d_c d_c^T - |d_c|^2 I)], d_c = com_c - o; then the
// centre of mass is o + S / M and the parallel-axis theorem moves Q_o to it:
// Q = Q_o - M (3 s s^T - |s|^2 I), s = S / M (the traceless quadrupole about
// the centre of mass, reading R3).  Every |d_c| and |s| is below the cell's
// diagonal, so no term is much larger than the result.
// kF32Q: the quadrupole is only needed by the FP32 walk, so it is summed in
// FP32 on the hi/lo records (d_c good to ~1e-7 relative); mass and centre of
// mass stay FP64.  On GB300 FP64 instructions cost 64 times FP32 ones.
// Running sums of one cell's moments about its first child's position o.
struct MomSums {
    double M, sx, sy, sz;   // mass and sum of M_c d_c (FP64)
    double q[6];            // quadrupole about o (FP64 form)
    float qf[6];            // quadrupole about o (FP32 form)
};

__device__ __forceinline__ void mom_zero(MomSums& S) {
    S.M = S.sx = S.sy = S.sz = 0.0;
#pragma unroll
    for (int j = 0; j < 6; j++) {
        S.q[j] = 0.0;
        S.qf[j] = 0.f;
    }
}

// Adds child entry c (a particle leaf or a finished deeper cell).
template <bool kF32Q>
__device__ __forceinline__ void mom_add(const GravRecArgs& A, int c, double ox, double oy, double oz,
                                        float4 h0, float4 l0, MomSums& S) {
    const double4_32a a = A.d_a[c];
    const bool leaf = __double_as_longlong(a.w) < 0;   // leaf records hold -m (m >= 0)
    const double mc = leaf ? -a.w : A.d_q0[c].x;
    const double dx = a.x - ox, dy = a.y - oy, dz = a.z - oz;
    S.M += mc;
    S.sx = fma(mc, dx, S.sx);
    S.sy = fma(mc, dy, S.sy);
    S.sz = fma(mc, dz, S.sz);
    if (kF32Q) {
        const float4 h = A.ra[c], l = A.rb[c];
        const float fx = (h.x - h0.x) + (l.x - l0.x);
        const float fy = (h.y - h0.y) + (l.y - l0.y);
        const float fz = (h.z - h0.z) + (h.w - h0.w);
        float fm;
        if (leaf) {
            fm = -l.z;
        } else {
            const float4 c0 = A.rq0[c], c1 = A.rq1[c];
            fm = c0.x;
            S.qf[0] += c0.y; S.qf[1] += c0.z; S.qf[2] += c0.w;
            S.qf[3] += c1.x; S.qf[4] += c1.y; S.qf[5] += c1.z;
        }
        const float d2 = fmaf(fz, fz, fmaf(fy, fy, fx * fx));
        const float m3x = 3.f * fm * fx, m3y = 3.f * fm * fy;
        S.qf[0] += fmaf(m3x, fx, -fm * d2);
        S.qf[1] += fmaf(m3y, fy, -fm * d2);
        S.qf[2] += fmaf(3.f * fm * fz, fz, -fm * d2);
        S.qf[3] += m3x * fy;
        S.qf[4] += m3x * fz;
        S.qf[5] += m3y * fz;
    } else {
        if (!leaf) {
            const double4_32a c0 = A.d_q0[c], c1 = A.d_q1[c];
            S.q[0] += c0.y; S.q[1] += c0.z; S.q[2] += c0.w;
            S.q[3] += c1.x; S.q[4] += c1.y; S.q[5] += c1.z;
        }
        const double d2 = dx * dx + dy * dy + dz * dz;
        S.q[0] += mc * (3.0 * dx * dx - d2);
        S.q[1] += mc * (3.0 * dy * dy - d2);
        S.q[2] += mc * (3.0 * dz * dz - d2);
        S.q[3] += mc * (3.0 * dx * dy);
        S.q[4] += mc * (3.0 * dx * dz);
        S.q[5] += mc * (3.0 * dy * dz);
    }
}

// Levels shared by two Morton keys (3 bits a level below the unused top bit).
__device__ __forceinline__ int common_levels(uint64_t a, uint64_t b) {
    const uint64_t x = a ^ b;
    return x ? (__clzll((long long)x) - 1) / 3 : kMaxDepth;
}

// A depth-21 leaf group (members first..last share their key) stands in the
// insertion tree below a run of one-child cells that reaches depth 20 unless
// its parent cell, the deepest one holding another particle of the box, is
// at depth 20 itself.  Those one-child cells hold the group's members and
// are opened or accepted like any cell; of them the depth-20 one accepts
// first (narrowest, and the smallest for the inside rule), so the group's
// record carries that cell's width and corner.  Without such a cell the group
// is never accepted.
__device__ __forceinline__ bool group_has_chain(const GravRecArgs& A, int first, int last) {
    const int n = min(A.ctl->n_live, A.ncap);
    const uint64_t kf = A.key[first];
    const int b = A.box[first];
    int d = -1;   // depth of the group's parent cell
    if (first > 0 && A.box[first - 1] == b) d = max(d, common_levels(A.key[first - 1], kf));
    if (last + 1 < n && A.box[last + 1] == b) d = max(d, common_levels(kf, A.key[last + 1]));
    return d < kMaxDepth - 1;
}

// The cell's centre of mass, its quadrupole moved there, and its records.
template <bool kF32Q>
__device__ __forceinline__ void mom_finish(const GravRecArgs& A, int k, int depth, int end, double ox,
                                           double oy, double oz, MomSums& S) {
    const int first = A.e_first[k];
    // a leaf group's members are the entries k + 1 .. end - 1
    const bool group = depth == kMaxDepth;
    const bool chain = group && group_has_chain(A, first, first + (end - k - 2));
    const int v = chain ? kMaxDepth - 1 : depth;   // the depth whose cell the record describes
    const BoxP bp = A.boxes[A.box[first]];
    const double w = ldexp(bp.L, -v);
    const double lo = -0.5 * bp.L;
    double ix = 0.0, iy = 0.0, iz = 0.0;
    if (A.inside || !(S.M > 0.0)) cell_index(A.key[first], v, ix, iy, iz);
    double cx, cy, cz, ux, uy, uz;   // centre of mass and its offset from o
    if (S.M > 0.0) {
        const double iM = 1.0 / S.M;
        ux = S.sx * iM; uy = S.sy * iM; uz = S.sz * iM;
        cx = ox + ux; cy = oy + uy; cz = oz + uz;
    } else {
        // no source mass (test particles only): the geometric centre
        cx = lo + (ix + 0.5) * w; cy = lo + (iy + 0.5) * w; cz = lo + (iz + 0.5) * w;
        ux = uy = uz = 0.0;
    }
    if (kF32Q) {
        const float fx = (float)ux, fy = (float)uy, fz = (float)uz, fm = (float)S.M;
        const float d2 = fmaf(fz, fz, fmaf(fy, fy, fx * fx));
        S.qf[0] -= fm * fmaf(3.f * fx, fx, -d2);
        S.qf[1] -= fm * fmaf(3.f * fy, fy, -d2);
        S.qf[2] -= fm * fmaf(3.f * fz, fz, -d2);
        S.qf[3] -= 3.f * fm * fx * fy;
        S.qf[4] -= 3.f * fm * fx * fz;
        S.qf[5] -= 3.f * fm * fy * fz;
#pragma unroll
        for (int j = 0; j < 6; j++) S.q[j] = (double)S.qf[j];
    } else {
        const double d2 = ux * ux + uy * uy + uz * uz;
        S.q[0] -= S.M * (3.0 * ux * ux - d2);
        S.q[1] -= S.M * (3.0 * uy * uy - d2);
        S.q[2] -= S.M * (3.0 * uz * uz - d2);
        S.q[3] -= S.M * (3.0 * ux * uy);
        S.q[4] -= S.M * (3.0 * ux * uz);
        S.q[5] -= S.M * (3.0 * uy * uz);
    }
    const bool never = group && !chain;   // a leaf group with no one-child cell above it
    const double ww = w * w;
    A.d_a[k] = make_double4_32a(cx, cy, cz, never ? __longlong_as_double(0x7ff0000000000000ll) : ww);
    A.d_q0[k] = make_double4_32a(S.M, S.q[0], S.q[1], S.q[2]);
    A.d_q1[k] = make_double4_32a(S.q[3], S.q[4], S.q[5], w);
    double c0x = 0.0, c0y = 0.0, c0z = 0.0;
    if (A.inside) {
        // cell corner lo + i w, rounded as two separate operations
        c0x = __dadd_rn(lo, __dmul_rn(ix, w));
        c0y = __dadd_rn(lo, __dmul_rn(iy, w));
        c0z = __dadd_rn(lo, __dmul_rn(iz, w));
        A.d_c[k] = make_double4_32a(c0x, c0y, c0z, w);
    }
    if (A.fp32) {
        float hx, lx, hy, ly, hz, lz;
        split_hilo(cx, hx, lx);
        split_hilo(cy, hy, ly);
        split_hilo(cz, hz, lz);
        const float crit = never ? __int_as_float(0x7f800000) : (float)(ww * A.crit_scale);
        A.ra[k] = make_float4(hx, hy, hz, lz);
        A.rb[k] = make_float4(lx, ly, crit, __int_as_float(end));
        if (kF32Q) {
            A.rq0[k] = make_float4((float)S.M, S.qf[0], S.qf[1], S.qf[2]);
            A.rq1[k] = make_float4(S.qf[3], S.qf[4], S.qf[5], 0.f);
        } else {
            A.rq0[k] = make_float4((float)S.M, (float)S.q[0], (float)S.q[1], (float)S.q[2]);
            A.rq1[k] = make_float4((float)S.q[3], (float)S.q[4], (float)S.q[5], 0.f);
        }
        if (A.inside) {
            split_hilo(c0x, hx, lx);
            split_hilo(c0y, hy, ly);
            split_hilo(c0z, hz, lz);
            A.rc_hi[k] = make_float4(hx, hy, hz, (float)w);
            A.rc_lo[k] = make_float4(lx, ly, lz, 0.f);
        }
    }
}

// The cells of one depth.  A cell's moments come from its children (deeper
// cells, done by earlier launches, or particle leaves) in one pass: about the
// first child's position o, M = sum M_c, S = sum M_c d_c and
// Q_o = sum [Q_c + M_c (3 d_c d_c^T - |d_c|^2 I)], d_c = com_c - o; then the
// centre of mass is o + S / M and the parallel-axis theorem moves Q_o to it:
// Q = Q_o - M (3 s s^T - |s|^2 I), s = S / M (the traceless quadrupole about
// the centre of mass, reading R3).  Every |d_c| and |s| is below the cell's
// diagonal, so no term is much larger than the result.
// kF32Q: the quadrupole is only needed by the FP32 walk, so it is summed in
// FP32 on the hi/lo records (d_c good to ~1e-7 relative); mass and centre of
// mass stay FP64.  On GB300 FP64 instructions cost 64 times FP32 ones.
// A depth with few cells (the top of the tree, the deep close pairs) is
// latency-bound: there eight lanes take one cell, one child each from the
// octant table, and add their sums in a fixed butterfly order; a depth with
// many cells gives each thread one cell, which follows its children in
// pre-order.
constexpr int kWarpCells = 19456;   // up to 4 cells per warp of the launch grid

template <bool kF32Q>
__global__ void __launch_bounds__(256) k_moments_level(GravRecArgs A, const int32_t* __restrict__ lvl,
                                                       const int32_t* __restrict__ list, int depth) {
    const int cnt = lvl[depth], off = lvl[32 + depth];
    if (cnt <= kWarpCells && depth < kMaxDepth) {
        const int lane = threadIdx.x & 31, o = lane & 7;   // o: octant of this lane's child
        const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwg = (gridDim.x * blockDim.x) >> 5;
        for (int base = 4 * wg; base < cnt; base += 4 * nwg) {
            // a warp takes 4 cells; a group past the end still joins the shuffles
            const int g = base + (lane >> 3);
            const bool live = g < cnt;
            const int k = live ? list[off + g] : 0;
            MomSums S;
            mom_zero(S);
            double ox = 0.0, oy = 0.0, oz = 0.0;
            float4 h0 = make_float4(0.f, 0.f, 0.f, 0.f), l0 = h0;
            if (live) {
                const double4_32a a0 = A.d_a[k + 1];   // the first child is entry k + 1
                ox = a0.x; oy = a0.y; oz = a0.z;
                if (kF32Q) {
                    h0 = A.ra[k + 1];
                    l0 = A.rb[k + 1];
                }
                if ((A.e_cmask[k] >> o) & 1u) mom_add<kF32Q>(A, A.e_child[8 * (size_t)k + o], ox, oy, oz, h0, l0, S);
            }
#pragma unroll
            for (int x = 1; x < 8; x <<= 1) {
                S.M += __shfl_xor_sync(0xffffffffu, S.M, x);
                S.sx += __shfl_xor_sync(0xffffffffu, S.sx, x);
                S.sy += __shfl_xor_sync(0xffffffffu, S.sy, x);
                S.sz += __shfl_xor_sync(0xffffffffu, S.sz, x);
#pragma unroll
                for (int j = 0; j < 6; j++) {
                    if (kF32Q) S.qf[j] += __shfl_xor_sync(0xffffffffu, S.qf[j], x);
                    else S.q[j] += __shfl_xor_sync(0xffffffffu, S.q[j], x);
                }
            }
            if (live && o == 0) mom_finish<kF32Q>(A, k, depth, A.e_skip[k], ox, oy, oz, S);
        }
        return;
    }
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
        const int k = list[off + t];
        const int end = A.e_skip[k];
        const double4_32a a0 = A.d_a[k + 1];
        const double ox = a0.x, oy = a0.y, oz = a0.z;
        float4 h0 = make_float4(0.f, 0.f, 0.f, 0.f), l0 = h0;
        if (kF32Q) {
            h0 = A.ra[k + 1];
            l0 = A.rb[k + 1];
        }
        MomSums S;
        mom_zero(S);
        for (int c = k + 1; c < end; c = A.e_skip[c]) mom_add<kF32Q>(A, c, ox, oy, oz, h0, l0, S);
        mom_finish<kF32Q>(A, k, depth, end, ox, oy, oz, S);
    }
}

struct CollRecArgs {
    const double *x, *y, *z, *r;
    const int32_t* box;
    const uint64_t* key;
    const BoxP* boxes;
    const int32_t *e_first, *e_skip, *leaf_of, *e_count, *e_child;
    const uint32_t* e_cmask;
    int32_t* e_top;
    const int8_t* e_level;
    Rec4 ra, rb;
    const Ctl* ctl;
    int ecap, ncap, nbox;
    double rmax;
    float4* pbox = nullptr;   // box items (pairs lo, hi): slots, then runs of 32, then runs of 256
};

// Collision-search records (Sect. 5.2): per cell its geometric centre
// (hi/lo) and the opening radius (sqrt(3)/2) w + R_max of Eq. 3, rounded up;
// per leaf the particle's position (hi/lo), slot and radius (the search
// leaves skip implicitly to the next entry).
__global__ void __launch_bounds__(256) k_coll_records(CollRecArgs A) {
    const int E = min(A.ctl->n_entries, A.ecap);
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= E) return;
    const int v = A.e_level[k];
    const int first = A.e_first[k];
    if (v == 22) {
        float hx, lx, hy, ly, hz, lz;
        split_hilo(A.x[first], hx, lx);
        split_hilo(A.y[first], hy, ly);
        split_hilo(A.z[first], hz, lz);
        A.ra[k] = make_float4(hx, hy, hz, __int_as_float(~first));
        A.rb[k] = make_float4(lx, ly, lz, (float)A.r[first]);
        return;
    }
    const BoxP bp = A.boxes[A.box[first]];
    const double w = ldexp(bp.L, -v);
    const double lo = -0.5 * bp.L;
    double ix, iy, iz;
    cell_index(A.key[first], v, ix, iy, iz);
    float hx, lx, hy, ly, hz, lz;
    split_hilo(lo + (ix + 0.5) * w, hx, lx);
    split_hilo(lo + (iy + 0.5) * w, hy, ly);
    split_hilo(lo + (iz + 0.5) * w, hz, lz);
    const float h = __double2float_ru(0.8660254037844387 * w + A.rmax);
    A.ra[k] = make_float4(hx, hy, hz, h);
    A.rb[k] = make_float4(lx, ly, lz, __int_as_float(A.e_skip[k]));
    A.e_top[k] = first + A.e_count[k] - 1;   // particles below sit at slots first ..
}

// Collision records on the gravity tree, at the positions after the second
// drift (Sect. 5.2, with a tighter pruning volume than Eq. 3's sphere): the
// tree's cells still hold the same particles, and a cell records the
// axis-aligned box of its particles' current positions (lower corner rounded
// down, upper corner rounded up to FP32), so the search stays exact without a
// second sort and build.  A cell's record also holds the largest particle
// slot below it (ra.w), so a search from slot i skips subtrees whose pairs
// with i are examined from the other particle.  Leaves as in
// k_coll_records; a removed particle's leaf sits at +infinity and is never
// close.
// Boxes from particle ranges: a cell of the gravity tree holds the
// consecutive slots [first, first + count), so its box is the union of its
// particles' boxes, taken here from the fewest aligned runs that tile the
// range (single slots at its ends, runs of 32, 256 and 8192 slots).
// Minima and maxima are exact in any order, so the records equal those of a
// bottom-up merge over the children, in three launches instead of one per
// depth.  A box item is the pair (lo, hi): lo = lower corner and the largest
// live slot (int bits, -1 none), hi = upper corner; an item with no live
// particle is (+inf, -inf).
constexpr int kRunA = 32, kRunB = 256, kRunC = 8192;
constexpr int kRunsInB = kRunB / kRunA, kRunsInC = kRunC / kRunB;
static_assert(kRunsInC == 32, "a warp per run of 8192 slots");

struct BoxAcc {
    float lox, loy, loz, hix, hiy, hiz;
    int top;
};

__device__ __forceinline__ BoxAcc box_empty() {
    const float inf = __int_as_float(0x7f800000);
    return BoxAcc{inf, inf, inf, -inf, -inf, -inf, -1};
}

__device__ __forceinline__ void box_fold(BoxAcc& B, const BoxAcc& o) {
    B.lox = fminf(B.lox, o.lox); B.loy = fminf(B.loy, o.loy); B.loz = fminf(B.loz, o.loz);
    B.hix = fmaxf(B.hix, o.hix); B.hiy = fmaxf(B.hiy, o.hiy); B.hiz = fmaxf(B.hiz, o.hiz);
    B.top = max(B.top, o.top);
}

// Fold of the boxes of the lanes l with (l & ~(width - 1)) equal, width a
// power of two up to 32.
__device__ __forceinline__ void box_reduce(BoxAcc& B, int width) {
    for (int x = 1; x < width; x <<= 1) {
        BoxAcc o;
        o.lox = __shfl_xor_sync(0xffffffffu, B.lox, x);
        o.loy = __shfl_xor_sync(0xffffffffu, B.loy, x);
        o.loz = __shfl_xor_sync(0xffffffffu, B.loz, x);
        o.hix = __shfl_xor_sync(0xffffffffu, B.hix, x);
        o.hiy = __shfl_xor_sync(0xffffffffu, B.hiy, x);
        o.hiz = __shfl_xor_sync(0xffffffffu, B.hiz, x);
        o.top = __shfl_xor_sync(0xffffffffu, B.top, x);
        box_fold(B, o);
    }
}

__device__ __forceinline__ void item_put(float4* pbox, long long i, const BoxAcc& B) {
    pbox[2 * i] = make_float4(B.lox, B.loy, B.loz, __int_as_float(B.top));
    pbox[2 * i + 1] = make_float4(B.hix, B.hiy, B.hiz, 0.f);
}

__device__ __forceinline__ void item_fold(const float4* pbox, long long i, BoxAcc& B) {
    const float4 lo = pbox[2 * i], hi = pbox[2 * i + 1];
    B.lox = fminf(B.lox, lo.x); B.loy = fminf(B.loy, lo.y); B.loz = fminf(B.loz, lo.z);
    B.hix = fmaxf(B.hix, hi.x); B.hiy = fmaxf(B.hiy, hi.y); B.hiz = fmaxf(B.hiz, hi.z);
    B.top = max(B.top, __float_as_int(lo.w));
}

__device__ __forceinline__ void cell_put(const CollRecArgs& A, int k, const BoxAcc& B) {
    A.ra[k] = make_float4(B.lox, B.loy, B.loz, __int_as_float(B.top));
    A.rb[k] = make_float4(B.hix, B.hiy, B.hiz, __int_as_float(A.e_skip[k]));
}

// Collision records on the gravity tree, at the positions after the second
// drift (Sect. 5.2, with a tighter pruning volume than Eq. 3's sphere): the
// tree's cells still hold the same particles, and a cell records the
// axis-aligned box of its particles' current positions (lower corner rounded
// down, upper corner rounded up to FP32), so the search stays exact without a
// second sort and build.  A cell's record also holds the largest particle
// slot below it (ra.w), so a search from slot i skips subtrees whose pairs
// with i are examined from the other particle.  Leaves as in
// k_coll_records; a removed particle's leaf sits at +infinity and is never
// close.  This launch also writes the box items of every slot and of the
// runs of 32 and 256 slots (kRunB threads per block).
__global__ void __launch_bounds__(kRunB) k_aabb_leaves(CollRecArgs A) {
    __shared__ BoxAcc wbox[kRunsInB];
    const int n = min(A.ctl->n_live, A.ncap);
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    BoxAcc B = box_empty();
    if (p < n) {
        const int e = A.leaf_of[p];
        if (A.box[p] >= A.nbox) {
            const float inf = __int_as_float(0x7f800000);
            A.ra[e] = make_float4(inf, inf, inf, __int_as_float(~p));
            A.rb[e] = make_float4(0.f, 0.f, 0.f, (float)A.r[p]);
        } else {
            float hx, lx, hy, ly, hz, lz;
            split_hilo(A.x[p], hx, lx);
            split_hilo(A.y[p], hy, ly);
            split_hilo(A.z[p], hz, lz);
            A.ra[e] = make_float4(hx, hy, hz, __int_as_float(~p));
            A.rb[e] = make_float4(lx, ly, lz, (float)A.r[p]);
            // hi = x rounded to nearest, lo the sign of x - hi: x lies in
            // [hi, next float up] or [next float down, hi]
            const float inf = __int_as_float(0x7f800000);
            B.lox = lx < 0.f ? nextafterf(hx, -inf) : hx;
            B.hix = lx > 0.f ? nextafterf(hx, inf) : hx;
            B.loy = ly < 0.f ? nextafterf(hy, -inf) : hy;
            B.hiy = ly > 0.f ? nextafterf(hy, inf) : hy;
            B.loz = lz < 0.f ? nextafterf(hz, -inf) : hz;
            B.hiz = lz > 0.f ? nextafterf(hz, inf) : hz;
            B.top = p;
        }
        item_put(A.pbox, p, B);
    }
    box_reduce(B, kRunA);
    const int w = threadIdx.x / kRunA;
    if (threadIdx.x % kRunA == 0) {
        if (p < n) item_put(A.pbox, (long long)A.ncap + p / kRunA, B);
        wbox[w] = B;
    }
    __syncthreads();
    if (w == 0) {
        BoxAcc C = (threadIdx.x < kRunsInB) ? wbox[threadIdx.x] : box_empty();
        box_reduce(C, kRunsInB);
        const int nruns = (A.ncap + kRunA - 1) / kRunA;
        if (threadIdx.x == 0 && blockIdx.x * kRunB < n)
            item_put(A.pbox, (long long)A.ncap + nruns + blockIdx.x, C);
    }
}

// The aligned pieces of [lo, hi) (units of the finer run) at a coarser run
// of `ratio` finer ones: the finer runs before the first coarse boundary,
// the coarse runs [c0, c1), the finer runs from c1 * ratio on.
struct Split {
    int head_end, c0, c1, tail_begin;
};
__device__ __forceinline__ Split split_runs(int lo, int hi, int ratio) {
    Split S;
    S.head_end = min(hi, (lo + ratio - 1) / ratio * ratio);
    S.tail_begin = max(S.head_end, hi / ratio * ratio);
    S.c0 = S.head_end / ratio;
    S.c1 = S.tail_begin / ratio;
    return S;
}

// Box items of the runs of 8192 slots, from their 32 runs of 256 (a warp per
// run).
__global__ void __launch_bounds__(256) k_aabb_runs(CollRecArgs A) {
    const int n = min(A.ctl->n_live, A.ncap);
    const long long nA = (A.ncap + kRunA - 1) / kRunA, nB = (A.ncap + kRunB - 1) / kRunB;
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int c = w; (long long)c * kRunC < n; c += nw) {
        BoxAcc B = box_empty();
        const int q = c * kRunsInC + lane;   // its run of 256
        if ((long long)q * kRunB < n) item_fold(A.pbox, A.ncap + nA + q, B);
        box_reduce(B, 32);
        if (lane == 0) item_put(A.pbox, A.ncap + nA + nB + c, B);
    }
}

// Folds the items that tile slots [a, e), lane `lane` of 32 taking every
// 32nd one: slots and runs of 32 and 256 at both ends, runs of 8192 between.
// A cell of c slots needs at most 138 + c / 8192 items.
__device__ __forceinline__ void range_fold(const CollRecArgs& A, int a, int e, int lane, BoxAcc& B) {
    const long long nA = (A.ncap + kRunA - 1) / kRunA, nB = (A.ncap + kRunB - 1) / kRunB;
    const long long baseA = A.ncap, baseB = baseA + nA, baseC = baseB + nB;
    const Split s1 = split_runs(a, e, kRunA);                // slots | runs of 32
    const Split s2 = split_runs(s1.c0, s1.c1, kRunsInB);     // runs of 32 | runs of 256
    const Split s3 = split_runs(s2.c0, s2.c1, kRunsInC);     // runs of 256 | runs of 8192
    // seven pieces in turn, each (first item index, count); `off` carries
    // this lane's position from one piece into the next
    int off = lane;
    auto piece = [&](long long first, int count) {
#pragma unroll 1
        for (; off < count; off += 32) item_fold(A.pbox, first + off, B);
        off -= count;
    };
    piece(a, s1.head_end - a);
    piece(baseA + s1.c0, s2.head_end - s1.c0);
    piece(baseB + s2.c0, s3.head_end - s2.c0);
    piece(baseC + s3.c0, s3.c1 - s3.c0);
    piece(baseB + s3.tail_begin, s2.c1 - s3.tail_begin);
    piece(baseA + s2.tail_begin, s1.c1 - s2.tail_begin);
    piece(s1.tail_begin, e - s1.tail_begin);
}

// Every cell of the gravity build, in entry order (consecutive entries: the
// counts and first slots are read coalesced; particle leaves are skipped).
// A lane takes a cell of at most eight slots alone; larger cells are taken
// afterwards by the whole warp, one at a time.
__global__ void __launch_bounds__(256) k_aabb_cells(CollRecArgs A) {
    const int E = min(A.ctl->n_entries, A.ecap);
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int e0 = 32 * w; e0 < E; e0 += 32 * nw) {
        const int k = e0 + lane;
        const bool cell = k < E && A.e_level[k] < 22;   // 22 marks a particle leaf
        int a = 0, c = 0;
        if (cell) {
            a = A.e_first[k];
            c = A.e_count[k];
        }
        if (cell && c <= 8) {
            BoxAcc B = box_empty();
#pragma unroll 4
            for (int j = 0; j < c; j++) item_fold(A.pbox, a + j, B);
            cell_put(A, k, B);
        }
        unsigned big = __ballot_sync(0xffffffffu, cell && c > 8);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const int ab = __shfl_sync(0xffffffffu, a, src);
            const int cb = __shfl_sync(0xffffffffu, c, src);
            BoxAcc W = box_empty();
            range_fold(A, ab, ab + cb, lane, W);
            box_reduce(W, 32);
            if (lane == 0) cell_put(A, e0 + src, W);
        }
    }
}

}  // namespace

void build_topology(const Tree& T, const PSet& P, Ctl* ctl, const BoxP* boxes, const SimC& C,
                    cudaStream_t s) {
    const int n = T.cap_n;
    if (n <= 0) return;
    const int nb = ceil_div(n, 256);
    cudaMemsetAsync(T.mask, 0, sizeof(uint32_t) * n, s);
    if (C.nbox > 1)
        k_nodes<true><<<nb, 256, 0, s>>>(T.key, P.box, ctl, n, T.node_a, T.node_b, T.node_v, T.mask);
    else
        k_nodes<false><<<nb, 256, 0, s>>>(T.key, P.box, ctl, n, T.node_a, T.node_b, T.node_v,
                                          T.mask);
    k_entry_counts<<<nb, 256, 0, s>>>(T.mask, ctl, n, T.start);
    exclusive_scan_i32(T.start, n, &ctl->n_live, T.scan_part, &ctl->n_entries, s);
    cudaMemsetAsync(T.e_cmask, 0, sizeof(uint32_t) * T.cap_e, s);
    k_emit<<<nb, 256, 0, s>>>(T.mask, T.start, T.node_a, T.node_b, T.node_v, ctl, n, T.e_first,
                              T.e_count, T.e_skip, T.e_level, T.leaf_of, T.key, T.e_child, T.e_cmask);
    k_box_ranges<<<ceil_div(n > C.nbox + 1 ? n : C.nbox + 1, 256), 256, 0, s>>>(
        P.box, ctl, n, C.nbox, T.box_first);
    k_box_roots<<<ceil_div(C.nbox + 1, 256), 256, 0, s>>>(T.box_first, T.start, C.nbox, T.box_root);
}

namespace {

// Hilbert index of (x, y) on a 2^lv grid (the classic quadrant rotation
// walk, most significant level first).
__device__ __forceinline__ uint32_t hilbert2(uint32_t x, uint32_t y, int lv) {
    const uint32_t n = 1u << lv;
    uint32_t d = 0;
    for (uint32_t s = n >> 1; s > 0; s >>= 1) {
        const uint32_t rx = (x & s) ? 1u : 0u, ry = (y & s) ? 1u : 0u;
        d += s * s * ((3u * rx) ^ ry);
        if (ry == 0) {
            if (rx == 1) {
                x = n - 1 - x;
                y = n - 1 - y;
            }
            const uint32_t t = x;
            x = y;
            y = t;
        }
    }
    return d;
}

// Hilbert index of (x, y, z) on a 2^lv grid: the axes are turned into the
// curve's "transposed" form (Skilling 2004, AIP Conf. Proc. 707: inverse
// undo of the excess work, then Gray decoding), whose bits interleaved
// from the top give the index.
__device__ __forceinline__ uint32_t hilbert3(uint32_t x, uint32_t y, uint32_t z, int lv) {
    uint32_t c[3] = {x, y, z};
    const uint32_t m = 1u << (lv - 1);
    for (uint32_t q = m; q > 1; q >>= 1) {
        const uint32_t p = q - 1;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            if (c[a] & q) {
                c[0] ^= p;
            } else {
                const uint32_t t = (c[0] ^ c[a]) & p;
                c[0] ^= t;
                c[a] ^= t;
            }
        }
    }
    c[1] ^= c[0];
    c[2] ^= c[1];
    uint32_t t = 0;
    for (uint32_t q = m; q > 1; q >>= 1)
        if (c[2] & q) t ^= q - 1;
    uint32_t d = 0;
    for (int b = lv - 1; b >= 0; b--)
#pragma unroll
        for (int a = 0; a < 3; a++) d = (d << 1) | (((c[a] ^ t) >> b) & 1u);
    return d;
}

// Tile keys of the sorted slots: the box above a Hilbert key of the slot's
// integer coordinates (read back from its Morton key); value = the slot.
__global__ void __launch_bounds__(256) k_tile_keys(const uint64_t* __restrict__ key,
                                                   const int32_t* __restrict__ box,
                                                   const Ctl* __restrict__ ctl, int ncap, int mode,
                                                   uint64_t* __restrict__ tkey, uint32_t* __restrict__ tval) {
    const int n = min(ctl->n_live, ncap);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t k = key[i];
    const uint32_t ix = morton_compact3(k >> 2), iy = morton_compact3(k >> 1), iz = morton_compact3(k);
    const uint32_t h = mode == kTileHilbertXY ? hilbert2(ix >> 11, iy >> 11, 10)
                                              : hilbert3(ix >> 14, iy >> 14, iz >> 14, 7);
    tkey[i] = ((uint64_t)(uint32_t)box[i] << 21) | (uint64_t)h;
    tval[i] = (uint32_t)i;
}

}  // namespace

void build_tile_order(Tree& T, const PSet& P, Ctl* ctl, int mode, int box_bits, cudaStream_t s) {
    if (mode == kTileMorton || T.cap_n <= 0) {
        T.order = nullptr;
        return;
    }
    k_tile_keys<<<ceil_div(T.cap_n, 256), 256, 0, s>>>(T.key, P.box, ctl, T.cap_n, mode, T.tkey, T.tval);
    const int which = radix_sort(T.tkey, T.tval, T.tkey_alt, T.tval_alt, T.cap_n, &ctl->n_live,
                                 21 + box_bits, nullptr, 0, T.hist, &ctl->err, s);
    T.order = which ? T.tval_alt : T.tval;
}

void build_gravity_records(const Tree& T, const PSet& P, Ctl* ctl, const BoxP* boxes,
                           const SimC& C, bool fp64, cudaStream_t s, bool f32q) {
    const int n = T.cap_n;
    if (n <= 0) return;
    GravRecArgs A;
    A.x = P.x; A.y = P.y; A.z = P.z; A.m = P.m; A.box = P.box; A.id = P.id;
    A.has_test = C.has_test != 0;
    A.key = T.key; A.boxes = boxes;
    A.e_first = T.e_first; A.e_skip = T.e_skip; A.e_child = T.e_child;
    A.e_cmask = T.e_cmask; A.leaf_of = T.leaf_of; A.e_level = T.e_level;
    A.e_arrive = T.e_arrive;
    A.d_a = T.d_a; A.d_q0 = T.d_q0; A.d_q1 = T.d_q1; A.d_c = T.d_c;
    A.ra = T.ra; A.rb = T.rb; A.rq0 = T.rq0; A.rq1 = T.rq1; A.rc_hi = T.rc_hi; A.rc_lo = T.rc_lo;
    A.ctl = ctl;
    A.ncap = n;
    A.crit_scale = C.crit_scale;
    A.fp32 = !fp64;
    A.inside = C.theta2 > (1.0 / 3.0);
    k_leaf_records<<<ceil_div(n, 256), 256, 0, s>>>(A);
    cudaMemsetAsync(T.lvl, 0, sizeof(int32_t) * 96, s);
    const int ne = T.cap_e;
    k_level_count<<<ceil_div(ne, 256), 256, 0, s>>>(T.e_level, ctl, ne, T.lvl);
    k_level_offsets<<<1, 1, 0, s>>>(T.lvl);
    k_level_fill<<<ceil_div(ne, 256), 256, 0, s>>>(T.e_level, ctl, ne, T.lvl, T.e_arrive);
    const int grid = std::min(ceil_div(n, 256), 4 * 152);
    const bool q32 = f32q && !fp64;
    for (int d = kMaxDepth; d >= 0; d--) {
        if (q32) k_moments_level<true><<<grid, 256, 0, s>>>(A, T.lvl, T.e_arrive, d);
        else k_moments_level<false><<<grid, 256, 0, s>>>(A, T.lvl, T.e_arrive, d);
    }
}

void build_collision_records(const Tree& T, const PSet& P, Ctl* ctl, const BoxP* boxes,
                             const SimC& C, double rmax, cudaStream_t s) {
    CollRecArgs A;
    A.x = P.x; A.y = P.y; A.z = P.z; A.r = P.r;
    A.box = P.box; A.key = T.key; A.boxes = boxes;
    A.e_first = T.e_first; A.e_skip = T.e_skip; A.e_level = T.e_level; A.leaf_of = T.leaf_of;
    A.e_count = T.e_count; A.e_top = T.e_top; A.e_child = T.e_child; A.e_cmask = T.e_cmask;
    A.ra = T.ra; A.rb = T.rb; A.ctl = ctl; A.ecap = T.cap_e; A.rmax = rmax;
    A.ncap = T.cap_n; A.nbox = C.nbox;
    k_coll_records<<<ceil_div(T.cap_e, 256), 256, 0, s>>>(A);
}

void build_collision_aabb(const Tree& T, const PSet& P, Ctl* ctl, const BoxP* boxes, const SimC& C,
                          double rmax, cudaStream_t s) {
    CollRecArgs A;
    A.x = P.x; A.y = P.y; A.z = P.z; A.r = P.r;
    A.box = P.box; A.key = T.key; A.boxes = boxes;
    A.e_first = T.e_first; A.e_skip = T.e_skip; A.e_level = T.e_level; A.leaf_of = T.leaf_of;
    A.e_count = T.e_count; A.e_top = T.e_top; A.e_child = T.e_child; A.e_cmask = T.e_cmask;
    A.ra = T.ra; A.rb = T.rb; A.ctl = ctl; A.ecap = T.cap_e; A.rmax = rmax;
    A.ncap = T.cap_n; A.nbox = C.nbox;
    A.pbox = T.pbox;
    k_aabb_leaves<<<ceil_div(T.cap_n, kRunB), kRunB, 0, s>>>(A);
    k_aabb_runs<<<ceil_div(ceil_div(T.cap_n, kRunC), 8), 256, 0, s>>>(A);
    // a warp per 32 entries; the resident blocks (48 registers: 5 of 256 per SM)
    const int grid = std::min(ceil_div(T.cap_e, 256), 5 * 152);
    k_aabb_cells<<<grid, 256, 0, s>>>(A);
}

}  // namespace rb
