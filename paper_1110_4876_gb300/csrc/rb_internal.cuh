// rb_internal.cuh -- device-side data layout and launch helpers of librb.
//
// Layout in HBM (one simulation, all boxes concatenated):
//  * particles: two FP64 SoA sets (x, y, z, vx, vy, vz, m, r) plus the
//    global id and the box of each particle; every tree build gathers the
//    current set into the other one in Morton order, so the arrays stay
//    sorted and every walk reads them coalesced;
//  * tree: "entries" in pre-order (depth-first) order, one per branching
//    cell and one per particle leaf, each with a skip index (the entry after
//    its subtree) so a walk needs no stack;
//  * walk records: 32-byte float4 pairs per entry for the FP32 walk (centre
//    of mass as a hi/lo float pair per axis, so differences of nearby points
//    keep ~1e-7 relative accuracy), 32-byte double4 records for the FP64
//    walk, and the FP64 moments (M, centre of mass, traceless quadrupole).
#pragma once
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

namespace rb {

constexpr int kMaxDepth = 21;           // 21 bits per axis in a 63-bit Morton key
constexpr uint64_t kRemovedKey = ~0ull; // sorts after every valid key (bit 63 set)
constexpr int kCentralCode = 7 | (7 << 4) | (7 << 8);
constexpr int kEnd = 0x7fffffff;        // "walk finished" marker

// Per-box parameters (device array, one entry per box).
struct BoxP {
    double L;            // root cube side (= Lx = Ly = Lz)
    double Lx, Ly, Lz;   // box sides (periodic lengths)
    double shear_speed;  // (1.5 * Omega) * Lx for shear-periodic boxes, else 0
    double key_scale;    // (1 / L, rounded) x 2^21, for the fast path of the integer coordinates
    double hx, hy, hz;   // half sides Lx / 2, Ly / 2, Lz / 2 (exact)
    int base_id;         // global id of the box's particle 0
    int n_active;        // particles with id - base_id >= n_active exert no gravity
};

// Constants of a simulation, passed by value to kernels.
struct SimC {
    int nbox, nimg, ngx, ngy, ngz;
    int boundary, z_periodic, integrator, quadrupole;
    double G, theta, theta2, soft2, eps, dt, half_dt, t0, omega, omega_z;
    double crit_scale;   // 1 / theta^2 (FP32 criterion (w / theta)^2)
    int has_test;        // some particles are test particles (source mass 0)
    int eps_law;         // 0: constant eps; 1: eps = min(1, (|v_n| / eps_vc)^(-eps_p))
    int hold_pair;       // test hook: the queue's first pair never becomes ready
    double eps_vc, eps_p;
    // SEI drift coefficients for tau = dt / 2 (x, vx, vy) -> (x, y, vx, vy), and z
    double axx, axu, axv, ayx, ayu, ayv, aux, auu, auv, avx, avu, avv;
    double azz, azw, awz, aww;
};

// One FP64 particle set (structure of arrays).
struct PSet {
    double *x, *y, *z, *vx, *vy, *vz, *m, *r;
    int32_t* id;   // global id (box base + id within the box)
    int32_t* box;  // box index; nbox marks a particle removed by an open boundary
};

// Device control block (scalars written by kernels).
struct Ctl {
    long long step;            // steps since the last set_particles / set_time
    int n_live;                // live particles after the last sort
    int n_live_next;           // live particles counted by the keys kernel
    int n_entries;             // tree entries (cells + leaves) of the last build
    int pair_count;            // pairs found by the last search (may exceed capacity)
    int pair_n;                // pairs to resolve (0 when the search overflowed)
    int pair_ends;             // 2 * pair_n
    int pending;               // pairs not yet resolved
    int resolved;              // pairs that were approaching and were resolved
    int err;                   // error bits (kErr*)
    int req_count;             // learned-correction requests recorded by the last walk
    int sweep_items;           // plane sweep: trajectory extents of the last search
    int out_live;              // host exchange: live particles of the box read out
    int pad_;
    unsigned long long n_cell, n_leaf, n_mac, n_recheck;
    unsigned long long n_iter;        // warp iterations of the last FP32 walk (entries visited)
    unsigned long long n_visit;       // tree entries tested by the targets of the last collision search
    unsigned long long n_siter;       // warp iterations of the last collision search
    unsigned long long sweep_wbits;   // plane sweep: largest half extent (double bits)
};
constexpr int kErrNonFinite = 1;
constexpr int kErrPairOverflow = 2;
constexpr int kErrSweepLong = 4;    // a plane-sweep item met more than kMaxSweepScan extents
constexpr int kErrResolveStall = 8; // the resolution queue stopped filling (bounded wait gave up)
constexpr int kErrWalk = 16;        // a walk met an entry index outside the tree (malformed tree)
constexpr int kErrSortStall = 32;   // a radix pass's look-back stopped advancing (bounded wait gave up)
constexpr int kMaxSweepScan = 1 << 16;

// One ghost image of one box at the time of a walk or search (Sect. 2.3):
// the offset in FP64 and as hi/lo floats, and the image's y velocity offset.
struct ImgTab {
    double ox, oy, oz, dvy;
    float4 hi, lo;   // w unused
};

// Box items of the collision records on the gravity tree: one per slot and
// per run of 32, 256 and 8192 slots.
inline long long box_items(int cap_n) {
    return (long long)cap_n + (cap_n + 31) / 32 + (cap_n + 255) / 256 + (cap_n + 8191) / 8192;
}

// Tree and scratch buffers of one build (sized for capacity n).
// One of two float4 records that an entry keeps side by side, so that the
// pair read together (e.g. centre of mass hi and lo) is one 32-byte sector:
// a view with stride 2 over the interleaved array.
struct Rec4 {
    float4* p = nullptr;
    __host__ __device__ float4& operator[](long long i) const { return p[2 * i]; }
};

struct Tree {
    uint64_t *key, *key_alt;    // sort keys (ping-pong)
    uint32_t *idx, *idx_alt;    // sort values: slot in the unsorted set
    int32_t* sbox;              // box digit per unsorted slot (nbox for removed)
    uint32_t* hist;             // radix sort block histograms
    int32_t* scan_part;         // block partials of the entry scan
    uint32_t* mask;             // per particle: levels of cells starting there
    int32_t* start;             // per particle: first entry starting there (n + 1)
    int32_t *node_a, *node_b;   // per split: first particle of its cell (last: reps only)
    int8_t* node_v;             // per split: cell depth (+32 unless representative), -1 none
    int32_t *e_first, *e_count, *e_skip, *e_arrive;
    int32_t* e_child;           // per cell entry: the child entry of each octant (8 slots)
    uint32_t* e_cmask;          // per cell entry: octants that hold a child
    int32_t* e_top;             // collision records on spheres: largest particle slot below
    int8_t* e_level;            // depth of a cell; 22 marks a particle leaf
    int32_t* leaf_of;           // per particle: its leaf entry
    double *M, *cx, *cy, *cz, *Q;   // FP64 moments per entry (Q: 6 x cap, xx yy zz xy xz yz)
    // FP32 walk records (pairs ra/rb, rq0/rq1 interleaved).  Gravity: ra =
    // (x_hi, y_hi, z_hi, z_lo), rb = (x_lo, y_lo, -m for a leaf or
    // (w / theta)^2 for a cell, skip entry), so the hi/lo pairs that the walk
    // subtracts from the target sit in aligned register pairs.  The collision
    // records written over them later in the step have their own layout.
    Rec4 ra, rb, rq0, rq1;
    Rec4 rc_hi, rc_lo;              // FP32 cell corner (hi/lo) + width, inside test
    float4* pbox;                   // collision boxes of slots and slot runs (box_items(cap_n) pairs)
    double4_32a *d_a, *d_q0, *d_q1, *d_c;  // FP64 walk records (d_c: cell corner + width)
    int32_t *box_first, *box_root;  // per box, nbox + 1 each (box_root[nbox] = -1: removed particles)
    int32_t* lvl;                   // per-depth cell counts / offsets / cursors (96)
    ImgTab* img;                    // [box][image] offsets of the current walk or search (nbox + 1 rows)
    int32_t* tq;                    // tile queues of the walks (kTileQStride ints each)
    int nq;                         // number of tile queues (one per SM)
    int cap_n, cap_e;
    // Order in which the walks and the search take their targets, 32 per
    // tile: nullptr = the Morton order of the slots; otherwise the slots
    // sorted by a Hilbert key (built by build_tile_order for each tree).
    uint64_t *tkey, *tkey_alt;
    uint32_t *tval, *tval_alt;
    const uint32_t* order = nullptr;
};

// Target orders of the walk and search tiles (the values of RB_TILE_*).
enum { kTileMorton = 0, kTileHilbertXY = 1, kTileHilbertXYZ = 2 };

// Pairs and their resolution.
struct Pairs {
    uint64_t *key, *key_alt;
    uint32_t *val, *val_alt;   // unused payload for the sort
    uint64_t *ekey, *ekey_alt; // pair ends: particle slot (sort key)
    uint32_t *eval, *eval_alt; // pair ends: 2 * pair + side
    int32_t *prev_a, *prev_b;  // previous pair (queue order) of particle a / b, or -1
    int32_t *next_a, *next_b;  // next pair of particle a / b, or -1
    int32_t* wait;             // unresolved predecessors of each pair
    int32_t* queue;            // pairs in the order they became ready (resolution)
    int32_t* rcnt;             // queue counters: [0] slots written, [1] slots claimed
    int32_t* slot_of_id;       // global id -> slot in the current set
    uint32_t *hist, *ehist;
    int cap;
    bool sorted_alt = false;   // the last pair sort left the sorted keys in key_alt
    const uint64_t* sorted() const { return sorted_alt ? key_alt : key; }
};

// Plane-sweep items (trajectory x extents, Sect. 5.3) and their sort buffers.
struct Sweep {
    uint64_t *key, *key_alt;   // (box << 32) | quantised lower end
    uint32_t *val, *val_alt;   // (particle slot << 3) | copy
    uint32_t* hist;
    void* rec;                 // per sorted item: the particle's state (64 B)
    int cap, box_bits;         // cap = particles x (1 + nghost_x)
};

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

#ifdef __CUDACC__
// Source mass of Eq. 1: test particles (id past the box's n_active) exert
// no gravity.
__device__ __forceinline__ double source_mass(const BoxP& bp, int id, double m) {
    return id - bp.base_id < bp.n_active ? m : 0.0;
}

// Time after 2 * step + hs drift halves: t0 + h * (dt / 2).
__device__ __forceinline__ double time_of(const Ctl* ctl, double t0, double half_dt, int hs) {
    const double h = (double)(2 * ctl->step + hs);
    return __dadd_rn(t0, __dmul_rn(h, half_dt));
}

// Ghost image offset (gx Lx, gy Ly - gx s, gz Lz), evaluated without
// contraction (Sect. 2.3; shear reading: s = fmod(1.5 Omega Lx t, Ly)).
__device__ __forceinline__ void image_offset(const BoxP& bp, double s, int gx, int gy, int gz,
                                             double& ox, double& oy, double& oz) {
    ox = __dmul_rn((double)gx, bp.Lx);
    oy = __dsub_rn(__dmul_rn((double)gy, bp.Ly), __dmul_rn((double)gx, s));
    oz = __dmul_rn((double)gz, bp.Lz);
}

__device__ __forceinline__ double shear_offset(const BoxP& bp, double t) {
    return bp.shear_speed != 0.0 ? fmod(__dmul_rn(bp.shear_speed, t), bp.Ly) : 0.0;
}

// Morton key -> integer cell index of depth v along each axis.
__device__ __forceinline__ uint32_t morton_compact3(uint64_t x) {
    x &= 0x1249249249249249ull;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
    x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
    x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
    x = (x ^ (x >> 32)) & 0x1fffffull;
    return (uint32_t)x;
}
#endif

// ---- launch wrappers (implemented in the .cu files) ----
// rb_sort.cu
int radix_sort_passes(int key_bits, bool box_pass, int box_bits);
// Sorts (key, val) pairs stably by key bits [0, key_bits) and then, when
// box_digits is non-null, by box_digits[val] (bits [0, box_bits)).
// Ping-pongs between the two buffers; returns 0 if the result is in
// (k0, v0) and 1 if it is in (k1, v1).  hist holds radix_hist_words(ncap)
// words; ncap < 2^30.  A look-back wait that gives up sets kErrSortStall in
// *err (device memory).
int radix_sort(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, int ncap, const int* d_n,
               int key_bits, const int32_t* box_digits, int box_bits, uint32_t* hist, int* err,
               cudaStream_t s);
size_t radix_hist_words(int ncap);
void exclusive_scan_i32(int32_t* data, int n_cap, const int* d_n, int32_t* part, int32_t* total,
                        cudaStream_t s);
size_t scan_part_words(int ncap);

// rb_tree.cu
void build_topology(const Tree& T, const PSet& P, Ctl* ctl, const BoxP* boxes, const SimC& C,
                    cudaStream_t s);
// Tile order of the current tree (T.key sorted, P its particles): mode
// kTileMorton leaves T.order null; kTileHilbertXY sorts the slots by a
// 10-level 2D Hilbert key of (x, y) (thin sheets), kTileHilbertXYZ by a
// 7-level 3D Hilbert key, the box id above either; ties keep Morton order.
void build_tile_order(Tree& T, const PSet& P, Ctl* ctl, int mode, int box_bits, cudaStream_t s);
// Moments and walk records.  fp64: FP64 records only (FP64 walk, potential);
// otherwise FP64 and FP32 records, and with f32q the quadrupole is summed in
// FP32 (the FP64 quadrupole records then hold its FP32 values).
void build_gravity_records(const Tree& T, const PSet& P, Ctl* ctl, const BoxP* boxes,
                           const SimC& C, bool fp64, cudaStream_t s, bool f32q = false);
// Collision records on the tree of the last gravity build at the current
// positions (cells as FP32 boxes of their particles); for collision_search
// with aabb = true.
void build_collision_aabb(const Tree& T, const PSet& P, Ctl* ctl, const BoxP* boxes, const SimC& C,
                          double rmax, cudaStream_t s);
void build_collision_records(const Tree& T, const PSet& P, Ctl* ctl, const BoxP* boxes,
                             const SimC& C, double rmax, cudaStream_t s);

// rb_walk.cu
struct WalkOut {
    double *ax, *ay, *az, *phi;   // per sorted slot
    int32_t *ncell, *nleaf, *nmac;
};
// Optional recording of accepted cells with w/R > theta_lo (learned mode):
// requests (slot << 40) | (image code << 28) | entry, kept when a hash of
// the request is below thresh.
struct WalkRecord {
    uint64_t* req;
    int* count;
    int cap;
    float band_scale;   // (theta_lo / theta)^2
    uint32_t thresh, seed;
};
// Learned walk (walk mode 2): accepted cells with w/R > theta_lo get the
// network's residual added inside the walk; the number of corrected cells is
// added to ctl->req_count.
namespace mlp { struct Packed; }
struct WalkLearn {
    const mlp::Packed* w;   // inference weights (device)
    float band_scale;       // (theta_lo / theta)^2
};
// Ghost-image table (tab: nbox x images) at the time 2 step + hs half steps;
// returns the images per box.  Images in (gx, gy, gz) loop order, gz fastest.
// With tq given, the same launch also empties the nq tile queues of the
// next walk or search.
int build_image_table(const BoxP* boxes, const Ctl* ctl, const SimC& C, int half_step_offset, ImgTab* tab,
                      cudaStream_t s, int32_t* tq = nullptr, int nq = 0);
// Walk and search kernels take their block size (64, 128 or 256 threads)
// at run time; the autotuner picks it.  They run persistent blocks (as many
// as fit on the GPU at once) that take tiles of 32 consecutive targets from
// per-SM queues: queue q holds the q-th contiguous part of the Morton order,
// so the warps resident on one SM walk neighbouring targets and share the
// tree records they read in that SM's L1.  An empty queue's warps take
// tiles from the following queues.
constexpr int kMaxWalkBlock = 256;
constexpr int kTileQStride = 8;     // ints per queue counter (one 32-byte sector each)
constexpr int kMaxTileQueues = 512;
// Queries the residency of every walk and search kernel once (outside any
// stream capture); returns the number of SMs.
int walk_prepare();
// group (plain FP32 walk only): 0 runs the union walk over the warp's 32
// targets; 4 runs the group walk, whose mixed subtrees are walked by
// subgroups of 4 lanes.  Accepted sets do not depend on block or group.
void gravity_walk(const Tree& T, const PSet& P, Ctl* ctl, const BoxP* boxes, const SimC& C,
                  int walk_mode, int half_step_offset, const WalkOut& out, bool potential,
                  bool counts, cudaStream_t s, const WalkRecord* rec = nullptr, int block = 128,
                  const WalkLearn* learn = nullptr, int group = 0);
// aabb: the records of build_collision_aabb, with rmax the largest radius.
// count: the variant that adds the entries its targets test and its warp
// iterations to ctl->n_visit and ctl->n_siter.
void collision_search(const Tree& T, const PSet& P, Ctl* ctl, const BoxP* boxes, const SimC& C,
                      const Pairs& PR, int half_step_offset, cudaStream_t s, int block = 128,
                      bool aabb = false, double rmax = 0.0, bool count = false);

// rb_sweep.cu: plane-sweep search on set P at half-step offset hs; the
// canonical pair keys are appended to PR like the tree search's.
void sweep_search(const PSet& P, Ctl* ctl, const BoxP* boxes, const SimC& C, Sweep& S,
                  const Pairs& PR, int half_step_offset, int ncap, cudaStream_t s);

// rb_step.cu
void drift_keys(const PSet& P, const Tree& T, Ctl* ctl, const BoxP* boxes, const SimC& C,
                int ncap, int ndrift, int half_step_offset, const double* ax, const double* ay,
                const double* az, bool kick, cudaStream_t s);
void sort_and_permute(const PSet& src, const PSet& dst, Tree& T, Pairs& PR, Ctl* ctl,
                      const SimC& C, int ncap, int box_bits, cudaStream_t s);
void resolve_pairs(const PSet& P, Ctl* ctl, const BoxP* boxes, const SimC& C, Pairs& PR,
                   int half_step_offset, ImgTab* img, cudaStream_t s);
// Queries the resident blocks of the resolution queue once (outside any
// stream capture).
void resolve_prepare(int nsm);
// key_bits: bits of the largest pair key, 36 + the bits of the largest id
void sort_pairs(Pairs& PR, Ctl* ctl, cudaStream_t s, int key_bits = 60);
void energy_terms(const PSet& P, Ctl* ctl, const SimC& C, const double* phi, int box,
                  double* partials, int nparts, double* out7, cudaStream_t s);
void step_advance(Ctl* ctl, cudaStream_t s);
// Host exchange: the live particles of a box in id order (out: 8 arrays of
// at least the box's size; flags: one int per id, set for live ids; *count:
// the live count), and the slot layout of a freshly copied single box.
void particles_by_id(const PSet& P, const PSet& out, int box, int base, int ncap, int32_t* flags,
                     int nflags, int* count, cudaStream_t s);
void reset_slots(const PSet& P, int32_t* slot_of_id, int n, int ncap, int nbox, cudaStream_t s);
// out2[0]: bit 0 non-finite state, bit 1 negative mass or radius; out2[1]:
// the largest radius (double bits).  Particles [0, n) of P.
void check_particles(const PSet& P, int n, unsigned long long* out2, cudaStream_t s);
// The live count the keys kernel accumulated, dropped when no sort follows
// (the particles keep their slots; removed ones stay flagged).
void discard_live_count(Ctl* ctl, cudaStream_t s);

// rb_api.cu: message returned by rb_last_error(NULL) on this thread.
void set_global_error(const std::string& msg);

// rb_mlp.cu: learned far-field correction.
namespace mlp {
struct ReqArgs {
    const double *x, *y, *z, *m;
    const int32_t *id, *box;
    const BoxP* boxes;
    const Ctl* ctl;
    const uint64_t* key;               // sorted Morton keys of the tree
    const int32_t *e_first, *e_count;
    const int8_t* e_level;
    const double4_32a *d_a, *d_q0, *d_q1;
    const uint64_t* req;               // requests recorded by the walk
    const int* req_count;
    int req_cap;
    double G, t0, half_dt;
    int hs;                            // half-step offset of the walk's time
};
int padded_size();
void to_padded(const float* canonical, float* padded);
void from_padded(const float* padded, float* canonical);
cudaError_t grad_async(const void* wbf, const float* wf, const float* X, const float* Y,
                       const int32_t* idx, int n, int n_total, float* grad, float* loss,
                       cudaStream_t s);
void adam_async(float* w, float* m, float* v, const float* grad, void* wbf, float lr, int step,
                cudaStream_t s);
// FP32 debug gradient on canonical (unpadded) weights: G holds n x 9347
// per-row gradients, lrow n per-row squared errors.
cudaError_t grad_f32_async(const float* w, const float* X, const float* Y, int n, float* G, float* lrow,
                           float* grad, float* loss, cudaStream_t s);
void to_bf16_async(const float* w, void* wbf, cudaStream_t s);
void label_async(const ReqArgs& A, float* X, float* Y, int64_t* meta, int max_req, cudaStream_t s);
}  // namespace mlp
void clear_walk_stats(Ctl* ctl, cudaStream_t s);
void clear_search_stats(Ctl* ctl, cudaStream_t s);

}  // namespace rb
