// rb_api.cu -- the C ABI of librb: simulation state, device memory, the
// per-step CUDA graph and the test/measurement hooks.
//
// One step (Sect. 3, drift-kick-drift) is captured once into a CUDA graph:
//   drift dt/2 + boundaries + Morton keys -> sort -> gather -> tree ->
//   moments -> gravity walk -> kick + drift dt/2 + boundaries + keys ->
//   sort -> gather -> tree -> collision search -> pair sort -> resolution.
// Each gather moves the particles into the other SoA set, so two graphs are
// captured (one per starting set) and replayed alternately.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <random>
#include <string>
#include <utility>
#include <vector>

#include "rb.h"
#include "rb_internal.cuh"
#include "rb_mlp.cuh"

using namespace rb;

namespace {

thread_local std::string g_create_error;

}  // namespace

void rb::set_global_error(const std::string& msg) { g_create_error = msg; }

namespace {

struct BoxHost {
    double L[3];
    int64_t n = 0;       // particles given to rb_set_particles
    bool stale = false;  // the arrays below are out of date: the data went straight to the device
    std::vector<double> x, y, z, vx, vy, vz, m, r;
};

}  // namespace

struct rb_sim {
    rb_config cfg{};
    int nbox = 1;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<BoxHost> hb;
    std::vector<int64_t> base;  // first global id of each box
    SimC C{};
    // device state
    PSet P[2]{};
    int cur = 0;
    Tree T{};
    Pairs PR{};
    Ctl* ctl = nullptr;
    BoxP* d_boxes = nullptr;
    double *acc_x = nullptr, *acc_y = nullptr, *acc_z = nullptr, *phi = nullptr;
    int32_t *cnt_cell = nullptr, *cnt_leaf = nullptr, *cnt_mac = nullptr;
    int acc_set = -1;     // particle set the last gravity walk ran on
    double* e_part = nullptr;
    double* e_out = nullptr;
    int ncap = 0, ntot = 0, box_bits = 0;
    double rmax = 0.0;
    bool dirty = true, graphs_dirty = true;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int gafter[2] = {0, 0};
    std::vector<void*> allocs, pair_allocs;
    Sweep SW{};   // plane-sweep items (collisions == RB_COLL_SWEEP)
    int nsm = 0;                           // SMs of the device (tile queues of the walks)
    int64_t n_active = -1;                 // test particles: ids >= n_active per box
    int eps_law = 0;                       // restitution law (RB_EPS_*)
    int hold_pair = 0;                     // test hook (rb_debug_hold_pair)
    double eps_vc = 1.0, eps_p = 0.0;
    std::string err;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t ev_stage[13] = {};
    // a branch of the step graph: the tile order of the targets runs on `side`
    // beside the moments, which leave most of the GPU idle
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int profiling = 0;   // 1: stage events; 2: also the counting collision search
    int kernels_per_step = 0;
    float last_ms = 0.f;
    float stage_ms[12] = {};
    Ctl hctl{};
    // learned far-field correction
    float* mlp_w = nullptr;      // padded FP32 weights
    void* mlp_wbf = nullptr;     // padded BF16 weights
    mlp::Packed* mlp_pk = nullptr;  // inference layout read by the learned walk
    bool mlp_loaded = false;
    double theta_fb = 0.5;
    std::vector<void*> mlp_allocs;
    // launch shapes (threads per block) of the gravity walk and the search
    int walk_block = 128, search_block = 128;
    int walk_group = 0;   // FP32 walk: 0 union walk; 4 group walk (4-lane subgroups for mixed subtrees)
    int tile_order = kTileMorton;   // order in which walks and search take targets (kTile*)
    bool tuned = false;
};

namespace {

constexpr int kEnergyParts = 304;

int fail(rb_sim* s, int code, const std::string& msg) {
    if (s) s->err = msg; else g_create_error = msg;
    return code;
}

#define RB_CUDA(sim, call)                                                               \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(sim, RB_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Bits of the largest pair key (id_a << 36 | id_b << 12 | image code): ids
// are below the particle capacity, so the sort skips the digits above them.
int pair_key_bits(const rb_sim* s) {
    int b = 1;
    while (b < 24 && (1 << b) < s->ncap) b++;
    return std::min(60, 36 + b);
}

template <typename T>
int dalloc(rb_sim* s, T** p, size_t count, std::vector<void*>& list) {
    void* q = nullptr;
    cudaError_t e = cudaMallocAsync(&q, std::max<size_t>(count, 1) * sizeof(T), s->stream);
    if (e != cudaSuccess) return fail(s, RB_ERR_CUDA, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    list.push_back(q);
    *p = static_cast<T*>(q);
    return RB_OK;
}

void free_list(rb_sim* s, std::vector<void*>& list) {
    for (void* q : list) cudaFreeAsync(q, s->stream);
    list.clear();
}

void drop_graphs(rb_sim* s) {
    for (int k = 0; k < 2; k++)
        if (s->gexec[k]) {
            cudaGraphExecDestroy(s->gexec[k]);
            s->gexec[k] = nullptr;
        }
    s->graphs_dirty = true;
}

// SimC from the configuration.  The SEI drift coefficients are the exact
// solution of Hill's equations over tau = dt/2 (Sect. 3.3).
void make_constants(rb_sim* s) {
    const rb_config& c = s->cfg;
    SimC& C = s->C;
    C.nbox = s->nbox;
    C.boundary = c.boundary;
    C.z_periodic = c.z_periodic;
    C.integrator = c.integrator;
    C.quadrupole = c.quadrupole;
    C.ngx = c.boundary == RB_BC_OPEN ? 0 : c.nghost[0];
    C.ngy = c.boundary == RB_BC_OPEN ? 0 : c.nghost[1];
    C.ngz = (c.boundary == RB_BC_OPEN || !c.z_periodic) ? 0 : c.nghost[2];
    C.nimg = (2 * C.ngx + 1) * (2 * C.ngy + 1) * (2 * C.ngz + 1);
    C.has_test = s->n_active >= 0;
    C.eps_law = s->eps_law;
    C.hold_pair = s->hold_pair;
    C.eps_vc = s->eps_vc;
    C.eps_p = s->eps_p;
    C.G = c.G;
    C.theta = c.theta;
    C.theta2 = c.theta * c.theta;
    C.crit_scale = 1.0 / (c.theta * c.theta);
    C.soft2 = c.softening * c.softening;
    C.eps = c.eps_restitution;
    C.dt = c.dt;
    C.half_dt = 0.5 * c.dt;
    C.t0 = c.t0;
    C.omega = c.omega;
    C.omega_z = c.omega_z > 0.0 ? c.omega_z : c.omega;
    if (c.integrator == RB_INT_SEI) {
        const double O = C.omega, Oz = C.omega_z, tau = 0.5 * c.dt;
        const double ph = O * tau, co = std::cos(ph), si = std::sin(ph);
        const double phz = Oz * tau, cz = std::cos(phz), sz = std::sin(phz);
        C.axx = 4.0 - 3.0 * co; C.axu = si / O; C.axv = (2.0 / O) * (1.0 - co);
        C.ayx = 6.0 * (si - ph); C.ayu = -(2.0 / O) * (1.0 - co); C.ayv = (4.0 * si - 3.0 * ph) / O;
        C.aux = (3.0 * O) * si; C.auu = co; C.auv = 2.0 * si;
        C.avx = (6.0 * O) * (co - 1.0); C.avu = -2.0 * si; C.avv = 4.0 * co - 3.0;
        C.azz = cz; C.azw = sz / Oz; C.awz = -(Oz * sz); C.aww = cz;
    }
}

int box_params(rb_sim* s) {
    std::vector<BoxP> hb(s->nbox);
    for (int b = 0; b < s->nbox; b++) {
        BoxP& p = hb[b];
        memset(&p, 0, sizeof(p));
        p.L = s->hb[b].L[0];
        p.Lx = s->hb[b].L[0]; p.Ly = s->hb[b].L[1]; p.Lz = s->hb[b].L[2];
        p.key_scale = (1.0 / p.L) * 2097152.0;   // exact scaling of the rounded reciprocal
        p.hx = 0.5 * p.Lx; p.hy = 0.5 * p.Ly; p.hz = 0.5 * p.Lz;
        p.shear_speed = s->cfg.boundary == RB_BC_SHEAR ? (1.5 * s->cfg.omega) * p.Lx : 0.0;
        p.base_id = b < (int)s->base.size() ? (int)s->base[b] : 0;
        p.n_active = s->n_active < 0 ? 0x7fffffff : (int)std::min<int64_t>(s->n_active, 0x7fffffff);
    }
    RB_CUDA(s, cudaMemcpyAsync(s->d_boxes, hb.data(), sizeof(BoxP) * s->nbox, cudaMemcpyHostToDevice,
                               s->stream));
    return RB_OK;
}

int alloc_pairs(rb_sim* s, int cap) {
    free_list(s, s->pair_allocs);
    Pairs& R = s->PR;
    int32_t* keep_slot = R.slot_of_id;
    R.cap = cap;
    int rc = RB_OK;
    auto& L = s->pair_allocs;
    rc |= dalloc(s, &R.key, cap, L);
    rc |= dalloc(s, &R.key_alt, cap, L);
    rc |= dalloc(s, &R.val, cap, L);
    rc |= dalloc(s, &R.val_alt, cap, L);
    rc |= dalloc(s, &R.ekey, 2 * (size_t)cap, L);
    rc |= dalloc(s, &R.ekey_alt, 2 * (size_t)cap, L);
    rc |= dalloc(s, &R.eval, 2 * (size_t)cap, L);
    rc |= dalloc(s, &R.eval_alt, 2 * (size_t)cap, L);
    rc |= dalloc(s, &R.prev_a, cap, L);
    rc |= dalloc(s, &R.prev_b, cap, L);
    rc |= dalloc(s, &R.next_a, cap, L);
    rc |= dalloc(s, &R.next_b, cap, L);
    rc |= dalloc(s, &R.wait, cap, L);
    rc |= dalloc(s, &R.queue, cap, L);
    rc |= dalloc(s, &R.rcnt, 64, L);
    rc |= dalloc(s, &R.hist, radix_hist_words(cap), L);
    rc |= dalloc(s, &R.ehist, radix_hist_words(2 * cap), L);
    R.slot_of_id = keep_slot;
    return rc ? RB_ERR_CUDA : RB_OK;
}

// Allocate for capacity n and upload the staged boxes.
int upload(rb_sim* s) {
    int64_t tot = 0;
    s->base.assign(s->nbox, 0);
    for (int b = 0; b < s->nbox; b++) {
        s->base[b] = tot;
        tot += s->hb[b].n;
    }
    if (tot >= (1 << 24)) return fail(s, RB_ERR_ARG, "more than 2^24 - 1 particles");
    const int n = (int)tot;
    if (n > s->ncap || s->ncap == 0) {
        drop_graphs(s);   // the graphs hold the old buffers
        free_list(s, s->allocs);
        free_list(s, s->pair_allocs);
        const int cap = std::max(n, 1);
        const int ecap = 2 * cap;
        auto& L = s->allocs;
        int rc = RB_OK;
        for (int k = 0; k < 2; k++) {
            PSet& P = s->P[k];
            rc |= dalloc(s, &P.x, cap, L); rc |= dalloc(s, &P.y, cap, L); rc |= dalloc(s, &P.z, cap, L);
            rc |= dalloc(s, &P.vx, cap, L); rc |= dalloc(s, &P.vy, cap, L); rc |= dalloc(s, &P.vz, cap, L);
            rc |= dalloc(s, &P.m, cap, L); rc |= dalloc(s, &P.r, cap, L);
            rc |= dalloc(s, &P.id, cap, L); rc |= dalloc(s, &P.box, cap, L);
        }
        Tree& T = s->T;
        T = Tree{};
        T.cap_n = cap;
        T.cap_e = ecap;
        rc |= dalloc(s, &T.key, cap, L); rc |= dalloc(s, &T.key_alt, cap, L);
        rc |= dalloc(s, &T.tkey, cap, L); rc |= dalloc(s, &T.tkey_alt, cap, L);
        rc |= dalloc(s, &T.tval, cap, L); rc |= dalloc(s, &T.tval_alt, cap, L);
        rc |= dalloc(s, &T.idx, cap, L); rc |= dalloc(s, &T.idx_alt, cap, L);
        rc |= dalloc(s, &T.sbox, cap, L);
        rc |= dalloc(s, &T.hist, radix_hist_words(cap), L);
        rc |= dalloc(s, &T.scan_part, scan_part_words(cap), L);
        rc |= dalloc(s, &T.mask, cap, L);
        rc |= dalloc(s, &T.start, cap + 1, L);
        rc |= dalloc(s, &T.node_a, cap, L); rc |= dalloc(s, &T.node_b, cap, L);
        rc |= dalloc(s, &T.node_v, cap, L);
        rc |= dalloc(s, &T.e_first, ecap, L); rc |= dalloc(s, &T.e_count, ecap, L);
        rc |= dalloc(s, &T.e_skip, ecap, L); rc |= dalloc(s, &T.e_child, 8 * (size_t)ecap, L);
        rc |= dalloc(s, &T.e_cmask, ecap, L); rc |= dalloc(s, &T.e_arrive, ecap, L);
        rc |= dalloc(s, &T.e_top, ecap, L);
        rc |= dalloc(s, &T.e_level, ecap, L);
        rc |= dalloc(s, &T.leaf_of, cap, L);
        {
            // FP32 record pairs, each pair interleaved (Rec4)
            float4 *rab = nullptr, *rq = nullptr, *rcc = nullptr;
            rc |= dalloc(s, &rab, 2 * (size_t)ecap, L);
            rc |= dalloc(s, &rq, 2 * (size_t)ecap, L);
            rc |= dalloc(s, &rcc, 2 * (size_t)ecap, L);
            rc |= dalloc(s, &T.pbox, 2 * (size_t)box_items(cap), L);
            T.ra.p = rab; T.rb.p = rab ? rab + 1 : nullptr;
            T.rq0.p = rq; T.rq1.p = rq ? rq + 1 : nullptr;
            T.rc_hi.p = rcc; T.rc_lo.p = rcc ? rcc + 1 : nullptr;
        }
        rc |= dalloc(s, &T.d_a, ecap, L); rc |= dalloc(s, &T.d_q0, ecap, L);
        rc |= dalloc(s, &T.d_q1, ecap, L); rc |= dalloc(s, &T.d_c, ecap, L);
        rc |= dalloc(s, &T.box_first, s->nbox + 1, L);
        rc |= dalloc(s, &T.box_root, s->nbox + 1, L);
        rc |= dalloc(s, &T.lvl, 96, L);
        rc |= dalloc(s, &T.tq, kMaxTileQueues * kTileQStride, L);
        T.nq = s->nsm > 0 ? min(s->nsm, kMaxTileQueues) : 1;
        rc |= dalloc(s, &T.img, (size_t)(s->nbox + 1) * (2 * s->cfg.nghost[0] + 1) * (2 * s->cfg.nghost[1] + 1) *
                                    (2 * s->cfg.nghost[2] + 1), L);
        rc |= dalloc(s, &s->PR.slot_of_id, cap, L);
        rc |= dalloc(s, &s->acc_x, cap, L); rc |= dalloc(s, &s->acc_y, cap, L);
        rc |= dalloc(s, &s->acc_z, cap, L); rc |= dalloc(s, &s->phi, cap, L);
        rc |= dalloc(s, &s->cnt_cell, cap, L); rc |= dalloc(s, &s->cnt_leaf, cap, L);
        rc |= dalloc(s, &s->cnt_mac, cap, L);
        rc |= dalloc(s, &s->ctl, 1, L);
        rc |= dalloc(s, &s->d_boxes, s->nbox, L);
        rc |= dalloc(s, &s->e_part, 7 * kEnergyParts, L);
        rc |= dalloc(s, &s->e_out, 8, L);
        s->SW = Sweep{};
        if (s->cfg.collisions == RB_COLL_SWEEP) {
            const int ic = cap * (1 + (s->cfg.boundary == RB_BC_OPEN ? 0 : s->cfg.nghost[0]));
            rc |= dalloc(s, &s->SW.key, ic, L); rc |= dalloc(s, &s->SW.key_alt, ic, L);
            rc |= dalloc(s, &s->SW.val, ic, L); rc |= dalloc(s, &s->SW.val_alt, ic, L);
            rc |= dalloc(s, &s->SW.hist, radix_hist_words(ic), L);
            double4_32a* recs = nullptr;   // 64-byte records: two double4 each
            rc |= dalloc(s, &recs, 2 * (size_t)ic, L);
            s->SW.rec = recs;
            s->SW.cap = ic;
        }
        if (rc) return RB_ERR_CUDA;
        s->ncap = cap;
        // a freshly drawn dense sheet overlaps about one pair per particle
        if (alloc_pairs(s, 2 * cap + 4096) != RB_OK) return RB_ERR_CUDA;
    }
    s->ntot = n;
    // stage into one contiguous host buffer per field
    const int cap = s->ncap;
    std::vector<double> f(cap);
    std::vector<int32_t> ids(cap), bx(cap);
    double* dst[8] = {s->P[0].x, s->P[0].y, s->P[0].z, s->P[0].vx,
                      s->P[0].vy, s->P[0].vz, s->P[0].m, s->P[0].r};
    double rmax = 0.0;
    for (int fld = 0; fld < 8; fld++) {
        int k = 0;
        for (int b = 0; b < s->nbox; b++) {
            const BoxHost& h = s->hb[b];
            const std::vector<double>* src[8] = {&h.x, &h.y, &h.z, &h.vx, &h.vy, &h.vz, &h.m, &h.r};
            for (double v : *src[fld]) {
                f[k++] = v;
                if (fld == 7) rmax = std::max(rmax, v);
            }
        }
        for (; k < cap; k++) f[k] = 0.0;
        RB_CUDA(s, cudaMemcpyAsync(dst[fld], f.data(), sizeof(double) * cap, cudaMemcpyHostToDevice,
                                   s->stream));
        RB_CUDA(s, cudaStreamSynchronize(s->stream));
    }
    {
        int k = 0;
        for (int b = 0; b < s->nbox; b++)
            for (int64_t i = 0; i < s->hb[b].n; i++) {
                ids[k] = k;
                bx[k] = b;
                k++;
            }
        for (; k < cap; k++) {
            ids[k] = k;
            bx[k] = s->nbox;   // unused slot: treated as removed
        }
    }
    RB_CUDA(s, cudaMemcpyAsync(s->P[0].id, ids.data(), sizeof(int32_t) * cap, cudaMemcpyHostToDevice, s->stream));
    RB_CUDA(s, cudaMemcpyAsync(s->P[0].box, bx.data(), sizeof(int32_t) * cap, cudaMemcpyHostToDevice, s->stream));
    RB_CUDA(s, cudaMemcpyAsync(s->PR.slot_of_id, ids.data(), sizeof(int32_t) * cap, cudaMemcpyHostToDevice, s->stream));
    Ctl c{};
    c.n_live = n;
    RB_CUDA(s, cudaMemcpyAsync(s->ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, s->stream));
    RB_CUDA(s, cudaStreamSynchronize(s->stream));
    if (rmax != s->rmax) drop_graphs(s);   // R_max is a launch argument of the graphs
    s->rmax = rmax;
    s->cur = 0;
    s->acc_set = -1;
    s->box_bits = 0;
    if (s->nbox > 1) {
        while ((1 << s->box_bits) <= s->nbox) s->box_bits++;
    }
    s->SW.box_bits = s->box_bits;
    make_constants(s);
    if (box_params(s) != RB_OK) return RB_ERR_CUDA;
    s->dirty = false;
    return RB_OK;
}

WalkOut walk_out(rb_sim* s) {
    WalkOut o;
    o.ax = s->acc_x; o.ay = s->acc_y; o.az = s->acc_z; o.phi = s->phi;
    o.ncell = s->cnt_cell; o.nleaf = s->cnt_leaf; o.nmac = s->cnt_mac;
    return o;
}

// Learned-walk arguments: inference weights and the band w/R > theta_fb.
WalkLearn learn_args(const rb_sim* s) {
    const double r = s->theta_fb / s->cfg.theta;
    return WalkLearn{s->mlp_pk, (float)(r * r)};
}

// Arguments of the request kernels for the tree built on set c.
mlp::ReqArgs req_args(rb_sim* s, int c, int hs, const uint64_t* req, int cap) {
    mlp::ReqArgs A;
    const PSet& P = s->P[c];
    A.x = P.x; A.y = P.y; A.z = P.z; A.m = P.m; A.id = P.id; A.box = P.box;
    A.boxes = s->d_boxes; A.ctl = s->ctl; A.key = s->T.key;
    A.e_first = s->T.e_first; A.e_count = s->T.e_count; A.e_level = s->T.e_level;
    A.d_a = s->T.d_a; A.d_q0 = s->T.d_q0; A.d_q1 = s->T.d_q1;
    A.req = req; A.req_count = &s->ctl->req_count; A.req_cap = cap;
    A.G = s->C.G; A.t0 = s->C.t0; A.half_dt = s->C.half_dt; A.hs = hs;
    return A;
}

// Stage marker: an event record node in the step graph when profiling.
void mark(rb_sim* s, int k) {
    // External: a real event record node (inside a capture a plain record is
    // only an ordering marker)
    if (s->profiling) cudaEventRecordWithFlags(s->ev_stage[k], s->stream, cudaEventRecordExternal);
}

// The launches of one step starting from particle set p; returns the set
// that holds the particles afterwards.
int record_step(rb_sim* s, int p) {
    cudaStream_t st = s->stream;
    cudaMemsetAsync(&s->ctl->pair_count, 0, sizeof(int), st);
    cudaMemsetAsync(&s->ctl->err, 0, sizeof(int), st);
    clear_walk_stats(s->ctl, st);
    int c = p;
    mark(s, 0);
    if (s->cfg.gravity) {
        drift_keys(s->P[c], s->T, s->ctl, s->d_boxes, s->C, s->ncap, 1, 1, nullptr, nullptr, nullptr,
                   false, st);
        mark(s, 1);
        sort_and_permute(s->P[c], s->P[1 - c], s->T, s->PR, s->ctl, s->C, s->ncap, s->box_bits, st);
        c = 1 - c;
        mark(s, 2);
        build_topology(s->T, s->P[c], s->ctl, s->d_boxes, s->C, st);
        // the tile order reads the sorted keys and writes only its own
        // arrays: it runs on the side stream while the moments run here
        cudaEventRecord(s->ev_fork, st);
        cudaStreamWaitEvent(s->side, s->ev_fork, 0);
        build_tile_order(s->T, s->P[c], s->ctl, s->tile_order, s->box_bits, s->side);
        cudaEventRecord(s->ev_join, s->side);
        mark(s, 3);
        build_gravity_records(s->T, s->P[c], s->ctl, s->d_boxes, s->C, s->cfg.walk == RB_WALK_FP64, st, true);
        cudaStreamWaitEvent(st, s->ev_join, 0);
        mark(s, 4);
        if (s->cfg.walk == RB_WALK_FP32_LEARNED) {
            // walk at theta; accepted cells with w/R > theta_fb get the
            // network's residual inside the walk
            cudaMemsetAsync(&s->ctl->req_count, 0, sizeof(int), st);
            const WalkLearn L = learn_args(s);
            gravity_walk(s->T, s->P[c], s->ctl, s->d_boxes, s->C, RB_WALK_FP32, 1, walk_out(s), false,
                         true, st, nullptr, s->walk_block, &L);
        } else {
            gravity_walk(s->T, s->P[c], s->ctl, s->d_boxes, s->C, s->cfg.walk, 1, walk_out(s), false,
                         true, st, nullptr, s->walk_block, nullptr, s->walk_group);
        }
        mark(s, 5);
        drift_keys(s->P[c], s->T, s->ctl, s->d_boxes, s->C, s->ncap, 1, 2, s->acc_x, s->acc_y,
                   s->acc_z, true, st);
    } else {
        drift_keys(s->P[c], s->T, s->ctl, s->d_boxes, s->C, s->ncap, 2, 1, nullptr, nullptr, nullptr,
                   false, st);
        for (int k = 1; k <= 5; k++) mark(s, k);
    }
    mark(s, 6);
    if (s->cfg.collisions == RB_COLL_SWEEP) {
        // plane sweep on the particles where they are: no collision tree
        discard_live_count(s->ctl, st);
        for (int k = 7; k <= 9; k++) mark(s, k);
        sweep_search(s->P[c], s->ctl, s->d_boxes, s->C, s->SW, s->PR, 2, s->ncap, st);
        mark(s, 10);
        sort_pairs(s->PR, s->ctl, st, pair_key_bits(s));
        mark(s, 11);
        resolve_pairs(s->P[c], s->ctl, s->d_boxes, s->C, s->PR, 2, s->T.img, st);
    } else if (s->cfg.collisions && s->cfg.gravity) {
        // the gravity tree still holds the same particles: boxes of their
        // current positions replace a second sort and build
        discard_live_count(s->ctl, st);
        mark(s, 7);
        mark(s, 8);
        build_collision_aabb(s->T, s->P[c], s->ctl, s->d_boxes, s->C, s->rmax, st);
        mark(s, 9);
        collision_search(s->T, s->P[c], s->ctl, s->d_boxes, s->C, s->PR, 2, st, s->search_block, true,
                         s->rmax, s->profiling == 2);
        mark(s, 10);
        sort_pairs(s->PR, s->ctl, st, pair_key_bits(s));
        mark(s, 11);
        resolve_pairs(s->P[c], s->ctl, s->d_boxes, s->C, s->PR, 2, s->T.img, st);
    } else if (s->cfg.collisions) {
        sort_and_permute(s->P[c], s->P[1 - c], s->T, s->PR, s->ctl, s->C, s->ncap, s->box_bits, st);
        c = 1 - c;
        mark(s, 7);
        build_topology(s->T, s->P[c], s->ctl, s->d_boxes, s->C, st);
        build_tile_order(s->T, s->P[c], s->ctl, s->tile_order, s->box_bits, st);
        mark(s, 8);
        build_collision_records(s->T, s->P[c], s->ctl, s->d_boxes, s->C, s->rmax, st);
        mark(s, 9);
        collision_search(s->T, s->P[c], s->ctl, s->d_boxes, s->C, s->PR, 2, st, s->search_block, false,
                         0.0, s->profiling == 2);
        mark(s, 10);
        sort_pairs(s->PR, s->ctl, st, pair_key_bits(s));
        mark(s, 11);
        resolve_pairs(s->P[c], s->ctl, s->d_boxes, s->C, s->PR, 2, s->T.img, st);
    } else {
        discard_live_count(s->ctl, st);   // no sort follows the last drift
        for (int k = 7; k <= 11; k++) mark(s, k);
    }
    mark(s, 12);
    step_advance(s->ctl, st);
    return c;
}

int capture_graphs(rb_sim* s) {
    drop_graphs(s);
    if (s->cfg.walk == RB_WALK_FP32_LEARNED && !s->mlp_loaded)
        return fail(s, RB_ERR_STATE, "the learned walk needs rb_load_mlp first");
    for (int p = 0; p < 2; p++) {
        cudaGraph_t g = nullptr;
        RB_CUDA(s, cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
        const int after = record_step(s, p);
        cudaError_t e = cudaStreamEndCapture(s->stream, &g);
        if (e != cudaSuccess) return fail(s, RB_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
        size_t nn = 0;
        cudaGraphGetNodes(g, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        cudaGraphGetNodes(g, nodes.data(), &nn);
        int nk = 0;
        for (auto nd : nodes) {
            cudaGraphNodeType ty;
            cudaGraphNodeGetType(nd, &ty);
            nk += ty == cudaGraphNodeTypeKernel;
        }
        s->kernels_per_step = nk;
        e = cudaGraphInstantiate(&s->gexec[p], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(s, RB_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
        s->gafter[p] = after;
    }
    s->graphs_dirty = false;
    return RB_OK;
}

__global__ void k_ctl_fresh(Ctl* ctl, int n) {
    Ctl c{};
    c.n_live = n;
    *ctl = c;
}

int read_ctl(rb_sim* s) {
    RB_CUDA(s, cudaMemcpyAsync(&s->hctl, s->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s->stream));
    RB_CUDA(s, cudaStreamSynchronize(s->stream));
    return RB_OK;
}

int clear_err(rb_sim* s) {
    RB_CUDA(s, cudaMemsetAsync(&s->ctl->err, 0, sizeof(int), s->stream));
    return RB_OK;
}

// Collision search + pair sort on set c at half-step offset hs; grows the
// pair buffer and searches again if it overflowed.  Resolves when asked.
int collide_with_retry(rb_sim* s, int c, int hs, bool resolve, bool aabb) {
    for (int attempt = 0; attempt < 2; attempt++) {
        RB_CUDA(s, cudaMemsetAsync(&s->ctl->pair_count, 0, sizeof(int), s->stream));
        clear_search_stats(s->ctl, s->stream);
        if (clear_err(s)) return RB_ERR_CUDA;
        if (s->cfg.collisions == RB_COLL_SWEEP)
            sweep_search(s->P[c], s->ctl, s->d_boxes, s->C, s->SW, s->PR, hs, s->ncap, s->stream);
        else
            collision_search(s->T, s->P[c], s->ctl, s->d_boxes, s->C, s->PR, hs, s->stream,
                             s->search_block, aabb, s->rmax, s->profiling == 2);
        sort_pairs(s->PR, s->ctl, s->stream, pair_key_bits(s));
        if (read_ctl(s)) return RB_ERR_CUDA;
        if (s->hctl.err & kErrSweepLong)
            return fail(s, RB_ERR_CAPACITY, "plane sweep: a trajectory overlaps more than 65536 others in x "
                                            "(use the tree detector)");
        if (s->hctl.err & kErrSortStall)
            return fail(s, RB_ERR_TIMEOUT, "radix sort: a bounded look-back wait gave up");
        if (s->hctl.pair_count <= s->PR.cap) {
            if (resolve) {
                resolve_pairs(s->P[c], s->ctl, s->d_boxes, s->C, s->PR, hs, s->T.img, s->stream);
                if (read_ctl(s)) return RB_ERR_CUDA;
                if (s->hctl.err & kErrResolveStall)
                    return fail(s, RB_ERR_TIMEOUT,
                                "collision resolution: a bounded wait for the ready queue gave up");
            }
            return RB_OK;
        }
        int cap = s->PR.cap;
        while (cap < s->hctl.pair_count) cap *= 2;
        if (alloc_pairs(s, cap + 4096) != RB_OK) return RB_ERR_CUDA;
        drop_graphs(s);
    }
    return fail(s, RB_ERR_CAPACITY, "collision pair buffer overflow persisted after growing");
}

int ensure_ready(rb_sim* s) {
    if (s->dirty) {
        int rc = upload(s);
        if (rc) return rc;
    }
    return RB_OK;
}

// Keys of the current positions (no drift), sort, gather, topology.
int rebuild_now(rb_sim* s) {
    const int c = s->cur;
    drift_keys(s->P[c], s->T, s->ctl, s->d_boxes, s->C, s->ncap, 0, 0, nullptr, nullptr, nullptr,
               false, s->stream);
    sort_and_permute(s->P[c], s->P[1 - c], s->T, s->PR, s->ctl, s->C, s->ncap, s->box_bits, s->stream);
    s->cur = 1 - c;
    build_topology(s->T, s->P[s->cur], s->ctl, s->d_boxes, s->C, s->stream);
    build_tile_order(s->T, s->P[s->cur], s->ctl, s->tile_order, s->box_bits, s->stream);
    return RB_OK;
}

int gravity_now(rb_sim* s, bool potential) {
    const bool learned = !potential && s->cfg.walk == RB_WALK_FP32_LEARNED;
    if (learned && !s->mlp_loaded) return fail(s, RB_ERR_STATE, "the learned walk needs rb_load_mlp first");
    rebuild_now(s);
    const bool fp64 = potential || s->cfg.walk == RB_WALK_FP64;
    build_gravity_records(s->T, s->P[s->cur], s->ctl, s->d_boxes, s->C, fp64, s->stream, true);
    clear_walk_stats(s->ctl, s->stream);
    if (learned) {
        cudaMemsetAsync(&s->ctl->req_count, 0, sizeof(int), s->stream);
        const WalkLearn L = learn_args(s);
        gravity_walk(s->T, s->P[s->cur], s->ctl, s->d_boxes, s->C, RB_WALK_FP32, 0, walk_out(s), false,
                     true, s->stream, nullptr, s->walk_block, &L);
    } else {
        gravity_walk(s->T, s->P[s->cur], s->ctl, s->d_boxes, s->C, fp64 ? RB_WALK_FP64 : s->cfg.walk, 0,
                     walk_out(s), potential, true, s->stream, nullptr, s->walk_block, nullptr,
                     s->walk_group);
    }
    s->acc_set = s->cur;
    RB_CUDA(s, cudaGetLastError());
    if (int rc = read_ctl(s)) return rc;
    if (s->hctl.err & kErrWalk)
        return fail(s, RB_ERR_STATE, "gravity walk: an entry index outside the tree (malformed tree)");
    if (s->hctl.err & kErrSortStall)
        return fail(s, RB_ERR_TIMEOUT, "radix sort: a bounded look-back wait gave up");
    return RB_OK;
}

template <typename T>
int d2h(rb_sim* s, std::vector<T>& v, const T* src, size_t n) {
    v.resize(std::max<size_t>(n, 1));
    RB_CUDA(s, cudaMemcpyAsync(v.data(), src, sizeof(T) * n, cudaMemcpyDeviceToHost, s->stream));
    RB_CUDA(s, cudaStreamSynchronize(s->stream));
    return RB_OK;
}

// (local id, slot) of the live particles of box b in set c, by id.
int live_slots(rb_sim* s, int c, int b, std::vector<std::pair<int64_t, int>>& out) {
    std::vector<int32_t> id, bx;
    if (d2h(s, id, s->P[c].id, s->ncap) || d2h(s, bx, s->P[c].box, s->ncap)) return RB_ERR_CUDA;
    out.clear();
    for (int i = 0; i < s->ncap; i++)
        if (bx[i] == b) out.emplace_back((int64_t)id[i] - s->base[b], i);
    std::sort(out.begin(), out.end());
    return RB_OK;
}

bool bad_box(rb_sim* s, int box) { return !s || box < 0 || box >= s->nbox; }

// The live particles of a box in id order: the device writes them in id
// order into the idle particle set, then each requested field is copied
// straight into the caller's array.  Ids removed by an open boundary leave
// gaps that are closed on the host.
int read_box(rb_sim* s, int box, int64_t cap, int64_t* n_out, double* const dst[8], int64_t* id) {
    const int nb = (int)s->hb[box].n;
    const PSet& out = s->P[1 - s->cur];
    int32_t* flags = s->T.start;   // scratch: ncap + 1 ints, free between steps
    particles_by_id(s->P[s->cur], out, box, (int)s->base[box], s->ncap, flags, nb, &s->ctl->out_live,
                    s->stream);
    // an open face (an open box, or the open z of a periodic or shearing box)
    // may have removed ids; otherwise every id of the box is live
    const bool may_remove = s->cfg.boundary == RB_BC_OPEN || !s->cfg.z_periodic;
    bool want = id != nullptr;
    for (int f = 0; f < 8; f++) want = want || dst[f] != nullptr;
    int live = nb;
    if (!want || (may_remove && cap < nb)) {
        if (may_remove) {
            if (read_ctl(s)) return RB_ERR_CUDA;
            live = s->hctl.out_live;
        }
        if (n_out) *n_out = live;
        if (!want) return RB_OK;   // a count query
    }
    if (live > cap) return fail(s, RB_ERR_ARG, "capacity too small");
    const double* src[8] = {out.x, out.y, out.z, out.vx, out.vy, out.vz, out.m, out.r};
    std::vector<int32_t> fl;
    if (cap >= nb) {
        // every id's entry straight into the caller's arrays; with removals
        // possible, the count read waits for these copies as well
        for (int f = 0; f < 8; f++)
            if (dst[f])
                RB_CUDA(s, cudaMemcpyAsync(dst[f], src[f], sizeof(double) * nb, cudaMemcpyDeviceToHost,
                                           s->stream));
        if (may_remove) {
            if (read_ctl(s)) return RB_ERR_CUDA;
            live = s->hctl.out_live;
        } else {
            RB_CUDA(s, cudaStreamSynchronize(s->stream));
        }
        if (n_out) *n_out = live;
        if (live == nb) {
            if (id)
                for (int k = 0; k < live; k++) id[k] = k;
            return RB_OK;
        }
        // removed ids leave gaps: keep the live entries, in id order
        if (d2h(s, fl, flags, nb)) return RB_ERR_CUDA;
        for (int f = 0; f < 8; f++) {
            if (!dst[f]) continue;
            int64_t k = 0;
            for (int j = 0; j < nb; j++)
                if (fl[j]) dst[f][k++] = dst[f][j];
        }
    } else {
        // fewer places than ids: through host buffers
        if (d2h(s, fl, flags, nb)) return RB_ERR_CUDA;
        std::vector<double> buf;
        for (int f = 0; f < 8; f++) {
            if (!dst[f]) continue;
            if (d2h(s, buf, src[f], nb)) return RB_ERR_CUDA;
            int64_t k = 0;
            for (int j = 0; j < nb; j++)
                if (fl[j]) dst[f][k++] = buf[j];
        }
    }
    if (id) {
        int64_t k = 0;
        for (int j = 0; j < nb; j++)
            if (fl[j]) id[k++] = j;
    }
    return RB_OK;
}

// The current particles of every box back into the host copies, before
// anything re-stages all boxes from the host (live particles, in id order).
int pull_to_host(rb_sim* s) {
    for (int b = 0; b < s->nbox; b++) {
        BoxHost& h = s->hb[b];
        int64_t n = 0;
        std::vector<double> f[8];
        for (auto& v : f) v.resize(std::max<int64_t>(h.n, 1));
        double* dst[8];
        for (int k = 0; k < 8; k++) dst[k] = f[k].data();
        int rc = read_box(s, b, h.n, &n, dst, nullptr);
        if (rc) return rc;
        std::vector<double>* hv[8] = {&h.x, &h.y, &h.z, &h.vx, &h.vy, &h.vz, &h.m, &h.r};
        for (int k = 0; k < 8; k++) hv[k]->assign(f[k].begin(), f[k].begin() + n);
        h.n = n;
        h.stale = false;
    }
    return RB_OK;
}

}  // namespace

extern "C" {

int rb_create(const rb_config* cfg, int nbox, void* cuda_stream, rb_sim** out) {
    if (!cfg || !out) return fail(nullptr, RB_ERR_ARG, "null argument");
    *out = nullptr;
    const rb_config& c = *cfg;
    if (nbox < 1 || nbox > 65535) return fail(nullptr, RB_ERR_ARG, "nbox must be in [1, 65535]");
    if (!(c.theta > 0.0)) return fail(nullptr, RB_ERR_ARG, "theta must be > 0");
    if (!(c.dt > 0.0)) return fail(nullptr, RB_ERR_ARG, "dt must be > 0");
    if (!(c.eps_restitution >= 0.0 && c.eps_restitution <= 1.0))
        return fail(nullptr, RB_ERR_ARG, "eps_restitution must be in [0, 1]");
    if (!(c.softening >= 0.0)) return fail(nullptr, RB_ERR_ARG, "softening must be >= 0");
    if (!(c.box[0] > 0.0 && c.box[1] > 0.0 && c.box[2] > 0.0) || c.box[1] > c.box[0] || c.box[2] > c.box[0])
        return fail(nullptr, RB_ERR_ARG, "box sides must be > 0 with box[1], box[2] <= box[0] (the root cube)");
    if (c.collisions < 0 || c.collisions > 2) return fail(nullptr, RB_ERR_ARG, "unknown collision detector");
    for (int a = 0; a < 3; a++)
        if (c.nghost[a] < 0 || c.nghost[a] > 7) return fail(nullptr, RB_ERR_ARG, "nghost must be in [0, 7]");
    if (c.boundary < 0 || c.boundary > 2) return fail(nullptr, RB_ERR_ARG, "unknown boundary");
    if (c.integrator < 0 || c.integrator > 1) return fail(nullptr, RB_ERR_ARG, "unknown integrator");
    if (c.walk < 0 || c.walk > 2) return fail(nullptr, RB_ERR_ARG, "unknown walk mode");
    if (c.integrator == RB_INT_SEI && !(c.omega > 0.0)) return fail(nullptr, RB_ERR_ARG, "SEI needs omega > 0");
    if (c.boundary == RB_BC_SHEAR && !(c.omega > 0.0)) return fail(nullptr, RB_ERR_ARG, "shear boundaries need omega > 0");
    if (c.nghost[2] > 0 && !c.z_periodic) return fail(nullptr, RB_ERR_ARG, "ghost boxes in z need z_periodic");
    if (c.z_periodic && c.boundary == RB_BC_OPEN) return fail(nullptr, RB_ERR_ARG, "z_periodic needs periodic or shear boundaries");
    for (int k = 0; k < 5; k++)
        if (c.reserved[k] != 0) return fail(nullptr, RB_ERR_ARG, "reserved fields must be zero");
    rb_sim* s = new rb_sim();
    s->cfg = c;
    s->nbox = nbox;
    s->hb.resize(nbox);
    for (auto& b : s->hb)
        for (int a = 0; a < 3; a++) b.L[a] = c.box[a];
    if (cuda_stream) {
        s->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete s;
            return fail(nullptr, RB_ERR_CUDA, "cudaStreamCreate failed");
        }
        s->own_stream = true;
    }
    s->nsm = walk_prepare();
    resolve_prepare(s->nsm);
    if (cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (s->ev_fork) cudaEventDestroy(s->ev_fork);
        if (s->side) cudaStreamDestroy(s->side);
        if (s->own_stream) cudaStreamDestroy(s->stream);
        delete s;
        return fail(nullptr, RB_ERR_CUDA, "cudaStreamCreate / cudaEventCreate failed");
    }
    cudaEventCreate(&s->ev0);
    cudaEventCreate(&s->ev1);
    for (auto& ev : s->ev_stage) cudaEventCreate(&ev);
    make_constants(s);
    *out = s;
    return RB_OK;
}

int rb_set_box(rb_sim* s, int box, const double L[3]) {
    if (bad_box(s, box) || !L) return fail(s, RB_ERR_ARG, "bad box or null L");
    if (!(L[0] > 0.0 && L[1] > 0.0 && L[2] > 0.0) || L[1] > L[0] || L[2] > L[0])
        return fail(s, RB_ERR_ARG, "box sides must be > 0 with L[1], L[2] <= L[0] (the root cube)");
    if (!s->dirty) {
        int rc = pull_to_host(s);
        if (rc) return rc;
    }
    for (int a = 0; a < 3; a++) s->hb[box].L[a] = L[a];
    s->dirty = true;
    return RB_OK;
}

int rb_set_particles(rb_sim* s, int box, int64_t n, const double* x, const double* y,
                     const double* z, const double* vx, const double* vy, const double* vz,
                     const double* m, const double* r) {
    if (bad_box(s, box) || n < 0) return fail(s, RB_ERR_ARG, "bad box or n < 0");
    if (n > 0 && (!x || !y || !z || !vx || !vy || !vz || !m || !r)) return fail(s, RB_ERR_ARG, "null array");
    BoxHost& h = s->hb[box];
    if (s->nbox == 1 && !s->dirty && n > 0 && n <= s->ncap && s->ctl) {
        // one box already on the device: copy the arrays straight into the
        // idle particle set, check them there, and switch to it (the current
        // state stays intact if the check fails)
        const int c = 1 - s->cur;
        const PSet& P = s->P[c];
        const double* src[8] = {x, y, z, vx, vy, vz, m, r};
        double* dst[8] = {P.x, P.y, P.z, P.vx, P.vy, P.vz, P.m, P.r};
        for (int f = 0; f < 8; f++)
            RB_CUDA(s, cudaMemcpyAsync(dst[f], src[f], sizeof(double) * n, cudaMemcpyHostToDevice, s->stream));
        unsigned long long* chk = reinterpret_cast<unsigned long long*>(s->e_out);
        check_particles(P, (int)n, chk, s->stream);
        unsigned long long hc[2] = {0, 0};
        RB_CUDA(s, cudaMemcpyAsync(hc, chk, sizeof(hc), cudaMemcpyDeviceToHost, s->stream));
        RB_CUDA(s, cudaStreamSynchronize(s->stream));
        if (hc[0] & 1ull) return fail(s, RB_ERR_NONFINITE, "non-finite particle state");
        if (hc[0] & 2ull) return fail(s, RB_ERR_ARG, "negative mass or radius");
        double rm = 0.0;
        memcpy(&rm, &hc[1], sizeof(rm));
        if (s->cfg.collisions && s->cfg.boundary != RB_BC_OPEN && 2.0 * rm >= std::min(h.L[0], h.L[1]))
            return fail(s, RB_ERR_ARG, "box side must exceed 2 max R");
        reset_slots(P, s->PR.slot_of_id, (int)n, s->ncap, s->nbox, s->stream);
        // the counters of a fresh state, written on the stream (no host wait:
        // the next call's work follows on the same stream)
        k_ctl_fresh<<<1, 1, 0, s->stream>>>(s->ctl, (int)n);
        RB_CUDA(s, cudaGetLastError());
        if (rm != s->rmax) drop_graphs(s);   // R_max is a launch argument of the graphs
        s->rmax = rm;
        s->cur = c;
        s->acc_set = -1;
        s->ntot = (int)n;
        s->base.assign(1, 0);
        h.n = n;
        h.stale = true;
        return RB_OK;
    }
    for (int64_t i = 0; i < n; i++) {
        if (!(std::isfinite(x[i]) && std::isfinite(y[i]) && std::isfinite(z[i]) && std::isfinite(vx[i]) &&
              std::isfinite(vy[i]) && std::isfinite(vz[i])))
            return fail(s, RB_ERR_NONFINITE, "non-finite particle state");
        if (!(m[i] >= 0.0) || !(r[i] >= 0.0)) return fail(s, RB_ERR_ARG, "negative mass or radius");
    }
    double rm = 0.0;
    for (int64_t i = 0; i < n; i++) rm = std::max(rm, r[i]);
    if (s->cfg.collisions && s->cfg.boundary != RB_BC_OPEN && 2.0 * rm >= std::min(h.L[0], h.L[1]))
        return fail(s, RB_ERR_ARG, "box side must exceed 2 max R");
    if (s->nbox > 1 && !s->dirty && s->ctl) {
        // the other boxes keep their current state (read back from the
        // device; ids that left through an open face are dropped)
        int rc = pull_to_host(s);
        if (rc) return rc;
    }
    h.x.assign(x, x + n); h.y.assign(y, y + n); h.z.assign(z, z + n);
    h.vx.assign(vx, vx + n); h.vy.assign(vy, vy + n); h.vz.assign(vz, vz + n);
    h.m.assign(m, m + n); h.r.assign(r, r + n);
    h.n = n;
    h.stale = false;
    s->dirty = true;
    return RB_OK;
}

int rb_step(rb_sim* s, int64_t nsteps) {
    if (!s || nsteps < 0) return fail(s, RB_ERR_ARG, "bad arguments");
    int rc = ensure_ready(s);
    if (rc) return rc;
    if (s->ntot == 0) return RB_OK;
    for (int64_t k = 0; k < nsteps; k++) {
        if (s->graphs_dirty && (rc = capture_graphs(s))) return rc;
        const int p = s->cur;
        RB_CUDA(s, cudaEventRecord(s->ev0, s->stream));
        RB_CUDA(s, cudaGraphLaunch(s->gexec[p], s->stream));
        RB_CUDA(s, cudaEventRecord(s->ev1, s->stream));
        if ((rc = read_ctl(s))) return rc;
        cudaEventElapsedTime(&s->last_ms, s->ev0, s->ev1);
        if (s->profiling)
            for (int q = 0; q < 12; q++)
                cudaEventElapsedTime(&s->stage_ms[q], s->ev_stage[q], s->ev_stage[q + 1]);
        s->cur = s->gafter[p];
        s->acc_set = s->cfg.gravity ? s->cur : -1;   // the walk's particle set (no second sort)
        if (s->hctl.err & kErrNonFinite)
            return fail(s, RB_ERR_NONFINITE, "a position became non-finite (or left the box by more than "
                                             "4096 box lengths in one drift half)");
        if (s->hctl.err & kErrWalk)
            return fail(s, RB_ERR_STATE, "gravity walk: an entry index outside the tree (malformed tree)");
        if (s->hctl.err & kErrSweepLong)
            return fail(s, RB_ERR_CAPACITY, "plane sweep: a trajectory overlaps more than 65536 others in x "
                                            "(use the tree detector)");
        if (s->hctl.err & kErrResolveStall)
            return fail(s, RB_ERR_TIMEOUT, "collision resolution: a bounded wait for the ready queue gave up");
        if (s->hctl.err & kErrSortStall)
            return fail(s, RB_ERR_TIMEOUT, "radix sort: a bounded look-back wait gave up");
        if (s->cfg.collisions && s->hctl.pair_count > s->PR.cap) {
            // the step ended before resolution: search again with a larger buffer
            const bool aabb = s->cfg.gravity && s->cfg.collisions == RB_COLL_TREE;
            if ((rc = collide_with_retry(s, s->cur, 0, true, aabb))) return rc;
        }
    }
    return RB_OK;
}

int rb_get_particles(rb_sim* s, int box, int64_t cap, int64_t* n_out, double* x, double* y,
                     double* z, double* vx, double* vy, double* vz, double* m, double* r,
                     int64_t* id) {
    if (bad_box(s, box)) return fail(s, RB_ERR_ARG, "bad box");
    int rc = ensure_ready(s);
    if (rc) return rc;
    double* dst[8] = {x, y, z, vx, vy, vz, m, r};
    return read_box(s, box, cap, n_out, dst, id);
}

int rb_compute_gravity(rb_sim* s) {
    if (!s) return fail(s, RB_ERR_ARG, "null sim");
    int rc = ensure_ready(s);
    if (rc) return rc;
    if (!s->cfg.gravity) return fail(s, RB_ERR_STATE, "gravity is off");
    if (s->ntot == 0) return RB_OK;
    return gravity_now(s, false);
}

int rb_get_accelerations(rb_sim* s, int box, int64_t cap, double* ax, double* ay, double* az) {
    if (bad_box(s, box)) return fail(s, RB_ERR_ARG, "bad box");
    if (s->acc_set < 0) return fail(s, RB_ERR_STATE, "no gravity walk yet");
    std::vector<std::pair<int64_t, int>> sl;
    if (live_slots(s, s->acc_set, box, sl)) return RB_ERR_CUDA;
    if ((int64_t)sl.size() > cap) return fail(s, RB_ERR_ARG, "capacity too small");
    const double* src[3] = {s->acc_x, s->acc_y, s->acc_z};
    double* dst[3] = {ax, ay, az};
    std::vector<double> buf;
    for (int f = 0; f < 3; f++) {
        if (!dst[f]) continue;
        if (d2h(s, buf, src[f], s->ncap)) return RB_ERR_CUDA;
        for (size_t k = 0; k < sl.size(); k++) dst[f][k] = buf[sl[k].second];
    }
    return RB_OK;
}

int rb_get_counts(rb_sim* s, int box, int64_t cap, int64_t* ncell, int64_t* nleaf, int64_t* nmac) {
    if (bad_box(s, box)) return fail(s, RB_ERR_ARG, "bad box");
    if (s->acc_set < 0) return fail(s, RB_ERR_STATE, "no gravity walk yet");
    std::vector<std::pair<int64_t, int>> sl;
    if (live_slots(s, s->acc_set, box, sl)) return RB_ERR_CUDA;
    if ((int64_t)sl.size() > cap) return fail(s, RB_ERR_ARG, "capacity too small");
    const int32_t* src[3] = {s->cnt_cell, s->cnt_leaf, s->cnt_mac};
    int64_t* dst[3] = {ncell, nleaf, nmac};
    std::vector<int32_t> buf;
    for (int f = 0; f < 3; f++) {
        if (!dst[f]) continue;
        if (d2h(s, buf, src[f], s->ncap)) return RB_ERR_CUDA;
        for (size_t k = 0; k < sl.size(); k++) dst[f][k] = buf[sl[k].second];
    }
    return RB_OK;
}

int rb_get_tree(rb_sim* s, int box, int64_t cap, int64_t* ncell, int32_t* depth, int64_t* count,
                double* M, double* com, double* Q, int64_t member_cap, int64_t* member_ids) {
    if (bad_box(s, box)) return fail(s, RB_ERR_ARG, "bad box");
    if (s->acc_set < 0) return fail(s, RB_ERR_STATE, "no gravity tree yet");
    if (read_ctl(s)) return RB_ERR_CUDA;
    const int E = s->hctl.n_entries;
    std::vector<int8_t> lev;
    std::vector<int32_t> first, cnt, skip, ids, roots;
    std::vector<double4_32a> da, q0, q1;
    if (d2h(s, lev, s->T.e_level, E) || d2h(s, first, s->T.e_first, E) || d2h(s, cnt, s->T.e_count, E) ||
        d2h(s, skip, s->T.e_skip, E) || d2h(s, ids, s->P[s->acc_set].id, s->ncap) ||
        d2h(s, roots, s->T.box_root, s->nbox) || d2h(s, da, s->T.d_a, E) || d2h(s, q0, s->T.d_q0, E) ||
        d2h(s, q1, s->T.d_q1, E))
        return RB_ERR_CUDA;
    int64_t k = 0, mk = 0;
    const int r0 = roots[box];
    if (r0 >= 0) {
        const int end = skip[r0];
        for (int e = r0; e < end; e++) {
            if (lev[e] == 22) continue;
            if (k < cap) {
                if (depth) depth[k] = lev[e];
                if (count) count[k] = cnt[e];
                if (M) M[k] = q0[e].x;
                if (com) { com[3 * k] = da[e].x; com[3 * k + 1] = da[e].y; com[3 * k + 2] = da[e].z; }
                if (Q) {
                    Q[6 * k] = q0[e].y; Q[6 * k + 1] = q0[e].z; Q[6 * k + 2] = q0[e].w;
                    Q[6 * k + 3] = q1[e].x; Q[6 * k + 4] = q1[e].y; Q[6 * k + 5] = q1[e].z;
                }
                if (member_ids && mk + cnt[e] <= member_cap)
                    for (int j = 0; j < cnt[e]; j++) member_ids[mk++] = ids[first[e] + j] - s->base[box];
            }
            k++;
        }
    }
    if (ncell) *ncell = k;
    return k > cap ? fail(s, RB_ERR_ARG, "capacity too small") : RB_OK;
}

int rb_detect_collisions(rb_sim* s) {
    if (!s) return fail(s, RB_ERR_ARG, "null sim");
    int rc = ensure_ready(s);
    if (rc) return rc;
    if (s->ntot == 0) return RB_OK;
    rebuild_now(s);
    if (s->cfg.collisions != RB_COLL_SWEEP)
        build_collision_records(s->T, s->P[s->cur], s->ctl, s->d_boxes, s->C, s->rmax, s->stream);
    return collide_with_retry(s, s->cur, 0, false, false);
}

int rb_get_pairs(rb_sim* s, int box, int64_t cap, int64_t* n, int64_t* id_a, int64_t* id_b,
                 int32_t* code) {
    if (bad_box(s, box)) return fail(s, RB_ERR_ARG, "bad box");
    if (read_ctl(s)) return RB_ERR_CUDA;
    const int np = s->hctl.pair_n;
    std::vector<uint64_t> keys;
    if (d2h(s, keys, s->PR.sorted(), np)) return RB_ERR_CUDA;
    const int64_t lo = s->base[box];
    const int64_t hi = lo + s->hb[box].n;
    int64_t k = 0;
    for (int i = 0; i < np; i++) {
        const int64_t a = (int64_t)(keys[i] >> 36);
        if (a < lo || a >= hi) continue;
        if (k < cap) {
            if (id_a) id_a[k] = a - lo;
            if (id_b) id_b[k] = (int64_t)((keys[i] >> 12) & 0xFFFFFFull) - lo;
            if (code) code[k] = (int32_t)(keys[i] & 0xFFFull);
        }
        k++;
    }
    if (n) *n = k;
    return k > cap ? fail(s, RB_ERR_ARG, "capacity too small") : RB_OK;
}

// K, U (SEI tidal + vertical), W, P of box `box` into h[0..6] (h[6] = n).
static int energy_sums(rb_sim* s, int box, double h[7]) {
    int rc = ensure_ready(s);
    if (rc) return rc;
    const double* phi = nullptr;
    if (s->cfg.gravity && s->ntot > 0) {
        if ((rc = gravity_now(s, true))) return rc;
        phi = s->phi;
    }
    energy_terms(s->P[s->cur], s->ctl, s->C, phi, box, s->e_part, kEnergyParts, s->e_out, s->stream);
    RB_CUDA(s, cudaMemcpyAsync(h, s->e_out, sizeof(double) * 7, cudaMemcpyDeviceToHost, s->stream));
    RB_CUDA(s, cudaStreamSynchronize(s->stream));
    return RB_OK;
}

int rb_energy(rb_sim* s, int box, double* E, double P[3]) {
    if (bad_box(s, box) || !E || !P) return fail(s, RB_ERR_ARG, "bad arguments");
    double h[8];
    int rc = energy_sums(s, box, h);
    if (rc) return rc;
    *E = h[0] + h[1] + h[2];
    P[0] = h[3]; P[1] = h[4]; P[2] = h[5];
    return RB_OK;
}

int rb_energy_terms(rb_sim* s, int box, double terms[6]) {
    if (bad_box(s, box) || !terms) return fail(s, RB_ERR_ARG, "bad arguments");
    double h[8];
    int rc = energy_sums(s, box, h);
    if (rc) return rc;
    for (int k = 0; k < 6; k++) terms[k] = h[k];
    return RB_OK;
}

int rb_set_pair_capacity(rb_sim* s, int64_t cap) {
    if (!s || cap < 1 || cap > 0x3fffffffll) return fail(s, RB_ERR_ARG, "bad pair capacity");
    int rc = ensure_ready(s);
    if (rc) return rc;
    drop_graphs(s);
    return alloc_pairs(s, (int)cap);
}

int rb_debug_hold_pair(rb_sim* s, int on) {
    if (!s) return fail(s, RB_ERR_ARG, "null simulation");
    s->hold_pair = on ? 1 : 0;
    make_constants(s);
    drop_graphs(s);
    return RB_OK;
}

int rb_set_time(rb_sim* s, double t) {
    if (!s || !std::isfinite(t)) return fail(s, RB_ERR_ARG, "bad time");
    s->cfg.t0 = t;
    make_constants(s);
    drop_graphs(s);
    if (!s->dirty && s->ctl) RB_CUDA(s, cudaMemsetAsync(&s->ctl->step, 0, sizeof(long long), s->stream));
    return RB_OK;
}

int rb_get_time(rb_sim* s, double* t) {
    if (!s || !t) return fail(s, RB_ERR_ARG, "bad arguments");
    long long step = 0;
    if (!s->dirty && s->ctl) {
        if (read_ctl(s)) return RB_ERR_CUDA;
        step = s->hctl.step;
    }
    *t = s->cfg.t0 + (double)(2 * step) * (0.5 * s->cfg.dt);
    return RB_OK;
}

int rb_stats(rb_sim* s, rb_stats_t* out) {
    if (!s || !out) return fail(s, RB_ERR_ARG, "bad arguments");
    memset(out, 0, sizeof(*out));
    if (s->dirty || !s->ctl) return RB_OK;
    if (read_ctl(s)) return RB_ERR_CUDA;
    const Ctl& c = s->hctl;
    out->steps = c.step;
    out->n_live = c.n_live;
    out->cells = c.n_entries > c.n_live ? c.n_entries - c.n_live : 0;   // one leaf per live particle
    out->pairs_found = c.pair_n;
    out->pairs_resolved = c.resolved;
    out->cell_interactions = (int64_t)c.n_cell;
    out->leaf_interactions = (int64_t)c.n_leaf;
    out->mac_tests = (int64_t)c.n_mac;
    out->fp64_rechecks = (int64_t)c.n_recheck;
    out->pair_capacity = s->PR.cap;
    out->t = s->cfg.t0 + (double)(2 * c.step) * (0.5 * s->cfg.dt);
    out->ms_last_step = s->last_ms;
    out->kernels_per_step = s->kernels_per_step;
    out->walk_block = s->walk_block;
    out->search_block = s->search_block;
    out->walk_group = s->walk_group;
    out->tile_order = s->tile_order;
    for (int q = 0; q < 12; q++) out->ms_stage[q] = s->stage_ms[q];
    out->corrections = s->cfg.walk == RB_WALK_FP32_LEARNED ? c.req_count : 0;
    out->warp_iterations = (int64_t)c.n_iter;
    out->search_visits = (int64_t)c.n_visit;
    out->search_iterations = (int64_t)c.n_siter;
    return RB_OK;
}

}  // extern "C"

namespace {

// Launch shapes chosen by rb_autotune, per (particle-count bucket, theta in
// thousandths, walk mode, batched boxes), shared by every simulation of the
// process.
struct TuneKey {
    int nbucket, theta_milli, walk, batched;
    bool operator<(const TuneKey& o) const {
        if (nbucket != o.nbucket) return nbucket < o.nbucket;
        if (theta_milli != o.theta_milli) return theta_milli < o.theta_milli;
        if (walk != o.walk) return walk < o.walk;
        return batched < o.batched;
    }
};
struct TuneShape {
    int walk_block, search_block, walk_group, tile_order;
};
std::map<TuneKey, TuneShape> g_tune_cache;
std::mutex g_tune_mutex;

TuneKey tune_key(const rb_sim* s) {
    int b = 0;
    while ((1LL << b) < (long long)std::max(s->ntot, 1)) b++;
    return TuneKey{b, (int)std::lround(s->cfg.theta * 1000.0), s->cfg.walk, s->nbox > 1 ? 1 : 0};
}

// Fastest of 3 repetitions (after one warm-up) of a launch sequence.
template <typename F>
float time_best(rb_sim* s, F&& launch) {
    launch();
    float best = 1e30f;
    for (int r = 0; r < 3; r++) {
        cudaEventRecord(s->ev0, s->stream);
        launch();
        cudaEventRecord(s->ev1, s->stream);
        cudaEventSynchronize(s->ev1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, s->ev0, s->ev1);
        best = std::min(best, ms);
    }
    return best;
}

}  // namespace

extern "C" {

int rb_autotune(rb_sim* s, int use_cache) {
    if (!s) return fail(s, RB_ERR_ARG, "null sim");
    int rc = ensure_ready(s);
    if (rc) return rc;
    if (s->ntot == 0) return RB_OK;
    const TuneKey key = tune_key(s);
    if (use_cache) {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            s->walk_block = it->second.walk_block;
            s->search_block = it->second.search_block;
            s->walk_group = it->second.walk_group;
            s->tile_order = it->second.tile_order;
            s->tuned = true;
            drop_graphs(s);
            return RB_OK;
        }
    }
    const int cand[3] = {64, 128, 256};
    int wb = s->walk_block, sb = s->search_block, wg = s->walk_group, to = s->tile_order;
    const bool fp64 = s->cfg.walk == RB_WALK_FP64;
    const bool learned = s->cfg.walk == RB_WALK_FP32_LEARNED && s->mlp_loaded;
    const WalkLearn L = learn_args(s);
    // the plain FP32 walk also chooses its warp shape: the union walk over 32
    // targets, or the group walk with 4-lane subgroups
    const bool grouped = !fp64 && !learned;
    const int gcand[2] = {0, 4};
    // every tile order is timed with the walk and the search it serves plus
    // the sort that builds it; the smallest sum wins
    const int ocand[3] = {kTileMorton, kTileHilbertXY, kTileHilbertXYZ};
    float best_total = 1e30f;
    for (int t : ocand) {
        s->tile_order = t;
        int wb_t = wb, sb_t = sb, wg_t = wg;
        float total = 0.f;
        if (s->cfg.gravity) {
            rebuild_now(s);
            if (t != kTileMorton)
                total += time_best(s, [&] {
                    build_tile_order(s->T, s->P[s->cur], s->ctl, t, s->box_bits, s->stream);
                });
            build_gravity_records(s->T, s->P[s->cur], s->ctl, s->d_boxes, s->C, fp64, s->stream, true);
            float best = 1e30f;
            for (int b : cand)
                for (int g : gcand) {
                    if (!grouped && g != gcand[0]) continue;
                    const float ms = time_best(s, [&] {
                        gravity_walk(s->T, s->P[s->cur], s->ctl, s->d_boxes, s->C,
                                     fp64 ? RB_WALK_FP64 : RB_WALK_FP32, 0, walk_out(s), false, false,
                                     s->stream, nullptr, b, learned ? &L : nullptr, g);
                    });
                    if (ms < best) { best = ms; wb_t = b; wg_t = grouped ? g : wg; }
                }
            total += best;
            s->acc_set = -1;   // the tuning walks left no consistent acceleration record
        }
        if (s->cfg.collisions == RB_COLL_TREE) {
            // the records the step uses: boxes on the gravity tree, or Eq. 3's
            // spheres on a collision tree when gravity is off
            const bool aabb = s->cfg.gravity != 0;
            rebuild_now(s);
            if (!s->cfg.gravity && t != kTileMorton)
                total += time_best(s, [&] {
                    build_tile_order(s->T, s->P[s->cur], s->ctl, t, s->box_bits, s->stream);
                });
            if (aabb) {
                build_gravity_records(s->T, s->P[s->cur], s->ctl, s->d_boxes, s->C, false, s->stream);
                build_collision_aabb(s->T, s->P[s->cur], s->ctl, s->d_boxes, s->C, s->rmax, s->stream);
            } else {
                build_collision_records(s->T, s->P[s->cur], s->ctl, s->d_boxes, s->C, s->rmax, s->stream);
            }
            float best = 1e30f;
            for (int b : cand) {
                const float ms = time_best(s, [&] {
                    cudaMemsetAsync(&s->ctl->pair_count, 0, sizeof(int), s->stream);
                    collision_search(s->T, s->P[s->cur], s->ctl, s->d_boxes, s->C, s->PR, 0, s->stream, b,
                                     aabb, s->rmax);
                });
                if (ms < best) { best = ms; sb_t = b; }
            }
            total += best;
            cudaMemsetAsync(&s->ctl->pair_n, 0, sizeof(int), s->stream);
        }
        if (total < best_total) {
            best_total = total;
            wb = wb_t; sb = sb_t; wg = wg_t; to = t;
        }
    }
    RB_CUDA(s, cudaStreamSynchronize(s->stream));
    RB_CUDA(s, cudaGetLastError());
    s->walk_block = wb;
    s->search_block = sb;
    s->walk_group = wg;
    s->tile_order = to;
    s->tuned = true;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = {wb, sb, wg, to};
    }
    drop_graphs(s);
    return RB_OK;
}

int rb_set_launch_shape(rb_sim* s, int walk_block, int search_block, int walk_group, int tile_order) {
    if (!s) return fail(s, RB_ERR_ARG, "null sim");
    const bool ok = (walk_block == 64 || walk_block == 128 || walk_block == 256) &&
                    (search_block == 64 || search_block == 128 || search_block == 256) &&
                    (walk_group == 0 || walk_group == 4) &&
                    (tile_order == RB_TILE_MORTON || tile_order == RB_TILE_HILBERT_XY ||
                     tile_order == RB_TILE_HILBERT_XYZ);
    if (!ok)
        return fail(s, RB_ERR_ARG,
                    "launch shapes: 64, 128 or 256 threads per block; walk group 0 or 4; tile order 0, 1 or 2");
    s->walk_block = walk_block;
    s->search_block = search_block;
    s->walk_group = walk_group;
    s->tile_order = tile_order;
    s->tuned = true;
    drop_graphs(s);
    return RB_OK;
}

int rb_set_n_active(rb_sim* s, int64_t n_active) {
    if (!s) return fail(s, RB_ERR_ARG, "null sim");
    s->n_active = n_active < 0 ? -1 : n_active;
    make_constants(s);
    drop_graphs(s);
    if (s->d_boxes && box_params(s) != RB_OK) return RB_ERR_CUDA;
    return RB_OK;
}

int rb_set_restitution(rb_sim* s, int law, double v_c, double p) {
    if (!s) return fail(s, RB_ERR_ARG, "null sim");
    if (law == RB_EPS_POWER && !(v_c > 0.0 && p >= 0.0 && std::isfinite(v_c) && std::isfinite(p)))
        return fail(s, RB_ERR_ARG, "power law needs v_c > 0 and p >= 0");
    if (law != RB_EPS_CONSTANT && law != RB_EPS_POWER) return fail(s, RB_ERR_ARG, "unknown restitution law");
    s->eps_law = law;
    s->eps_vc = law == RB_EPS_POWER ? v_c : 1.0;
    s->eps_p = law == RB_EPS_POWER ? p : 0.0;
    make_constants(s);
    drop_graphs(s);
    return RB_OK;
}

int rb_set_profiling(rb_sim* s, int on) {
    if (!s) return fail(s, RB_ERR_ARG, "null sim");
    if (on < 0 || on > 2) return fail(s, RB_ERR_ARG, "profiling level must be 0, 1 or 2");
    if (on != s->profiling) {
        s->profiling = on;
        drop_graphs(s);
    }
    return RB_OK;
}

void rb_destroy(rb_sim* s) {
    if (!s) return;
    drop_graphs(s);
    free_list(s, s->pair_allocs);
    free_list(s, s->allocs);
    free_list(s, s->mlp_allocs);
    cudaStreamSynchronize(s->stream);
    if (s->ev0) cudaEventDestroy(s->ev0);
    if (s->ev1) cudaEventDestroy(s->ev1);
    for (auto& ev : s->ev_stage)
        if (ev) cudaEventDestroy(ev);
    if (s->side) {
        cudaStreamSynchronize(s->side);
        cudaStreamDestroy(s->side);
    }
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    if (s->ev_join) cudaEventDestroy(s->ev_join);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
}

const char* rb_last_error(const rb_sim* s) {
    return s ? s->err.c_str() : g_create_error.c_str();
}

// ---- learned far-field correction ----

int rb_load_mlp(rb_sim* s, const float* w, int64_t nw, double theta_fallback) {
    if (!s || !w || nw != RB_MLP_PARAMS) return fail(s, RB_ERR_ARG, "expected 9347 weights");
    if (!(theta_fallback > 0.0) || theta_fallback > s->cfg.theta)
        return fail(s, RB_ERR_ARG, "theta_fallback must be in (0, theta]");
    for (int64_t i = 0; i < nw; i++)
        if (!std::isfinite(w[i])) return fail(s, RB_ERR_NONFINITE, "non-finite weight");
    const int np = mlp::padded_size();
    if (!s->mlp_w) {
        if (dalloc(s, &s->mlp_w, np, s->mlp_allocs)) return RB_ERR_CUDA;
        uint16_t* bf = nullptr;
        if (dalloc(s, &bf, np, s->mlp_allocs)) return RB_ERR_CUDA;
        s->mlp_wbf = bf;
        if (dalloc(s, &s->mlp_pk, 1, s->mlp_allocs)) return RB_ERR_CUDA;
    }
    std::vector<float> pad(np);
    mlp::to_padded(w, pad.data());
    RB_CUDA(s, cudaMemcpyAsync(s->mlp_w, pad.data(), sizeof(float) * np, cudaMemcpyHostToDevice, s->stream));
    mlp::to_bf16_async(s->mlp_w, s->mlp_wbf, s->stream);
    mlp::pack_async(s->mlp_w, s->mlp_pk, s->stream);
    RB_CUDA(s, cudaStreamSynchronize(s->stream));
    s->mlp_loaded = true;
    s->theta_fb = theta_fallback;
    drop_graphs(s);
    return RB_OK;
}

int rb_mlp_samples(rb_sim* s, double theta_hi, double theta_lo, double prob, uint64_t seed,
                   int64_t cap, int64_t* n_out, float* X, float* Y, int64_t* meta) {
    if (!s || !n_out || !(theta_hi > 0.0) || !(theta_lo > 0.0) || !(theta_lo < theta_hi) ||
        !(prob > 0.0) || cap < 1 || cap > 0x7fffffffll)
        return fail(s, RB_ERR_ARG, "bad sampling arguments");
    int rc = ensure_ready(s);
    if (rc) return rc;
    if (!s->cfg.gravity) return fail(s, RB_ERR_STATE, "gravity is off");
    *n_out = 0;
    if (s->ntot == 0) return RB_OK;
    rebuild_now(s);
    SimC C2 = s->C;
    C2.theta = theta_hi;
    C2.theta2 = theta_hi * theta_hi;
    C2.crit_scale = 1.0 / (theta_hi * theta_hi);
    build_gravity_records(s->T, s->P[s->cur], s->ctl, s->d_boxes, C2, false, s->stream);
    std::vector<void*> tmp;
    uint64_t* req = nullptr;
    float *dX = nullptr, *dY = nullptr;
    int64_t* dmeta = nullptr;
    if (dalloc(s, &req, cap, tmp) || dalloc(s, &dX, 12 * cap, tmp) || dalloc(s, &dY, 3 * cap, tmp) ||
        dalloc(s, &dmeta, 5 * cap, tmp)) {
        free_list(s, tmp);
        return RB_ERR_CUDA;
    }
    cudaMemsetAsync(&s->ctl->req_count, 0, sizeof(int), s->stream);
    const uint32_t thresh = prob >= 1.0 ? 0xffffffffu : (uint32_t)(prob * 4294967296.0);
    const WalkRecord rec{req, &s->ctl->req_count, (int)cap,
                         (float)((theta_lo / theta_hi) * (theta_lo / theta_hi)), thresh,
                         (uint32_t)(seed ^ (seed >> 32))};
    clear_walk_stats(s->ctl, s->stream);
    gravity_walk(s->T, s->P[s->cur], s->ctl, s->d_boxes, C2, RB_WALK_FP32, 0, walk_out(s), false, true,
                 s->stream, &rec);
    s->acc_set = s->cur;
    mlp::label_async(req_args(s, s->cur, 0, req, (int)cap), dX, dY, dmeta, (int)cap, s->stream);
    rc = read_ctl(s);
    const int64_t n = std::min<int64_t>(s->hctl.req_count, cap);
    if (!rc && n > 0) {
        if (X) cudaMemcpyAsync(X, dX, sizeof(float) * 12 * n, cudaMemcpyDeviceToHost, s->stream);
        if (Y) cudaMemcpyAsync(Y, dY, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, s->stream);
        if (meta) cudaMemcpyAsync(meta, dmeta, sizeof(int64_t) * 5 * n, cudaMemcpyDeviceToHost, s->stream);
        if (cudaStreamSynchronize(s->stream) != cudaSuccess) rc = fail(s, RB_ERR_CUDA, "sample copy failed");
    }
    free_list(s, tmp);
    cudaStreamSynchronize(s->stream);
    *n_out = n;
    return rc;
}

}  // extern "C"

// Standalone training and gradient entry points (no simulation).
namespace {

struct MlpBufs {
    cudaStream_t s = nullptr;
    bool own = false;
    std::vector<void*> ptrs;
    template <typename T>
    T* alloc(size_t n) {
        void* p = nullptr;
        if (cudaMallocAsync(&p, std::max<size_t>(n, 1) * sizeof(T), s) != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        return static_cast<T*>(p);
    }
    ~MlpBufs() {
        for (void* p : ptrs) cudaFreeAsync(p, s);
        cudaStreamSynchronize(s);
        if (own) cudaStreamDestroy(s);
    }
};

}  // namespace

extern "C" {

int rb_mlp_grad(const float* w, const float* X, const float* Y, int64_t n, float* grad, float* loss,
                void* cuda_stream) {
    if (!w || !X || !Y || n < 1 || n > 0x7fffffffll || !grad) {
        g_create_error = "rb_mlp_grad: bad arguments";
        return RB_ERR_ARG;
    }
    MlpBufs B;
    B.s = static_cast<cudaStream_t>(cuda_stream);
    if (!B.s) {
        cudaStreamCreateWithFlags(&B.s, cudaStreamNonBlocking);
        B.own = true;
    }
    const int np = mlp::padded_size();
    float* dw = B.alloc<float>(np);
    uint16_t* dwb = B.alloc<uint16_t>(np);
    float* dX = B.alloc<float>(12 * n);
    float* dY = B.alloc<float>(3 * n);
    int32_t* didx = B.alloc<int32_t>(n);
    float* dg = B.alloc<float>(np);
    float* dl = B.alloc<float>(1);
    if (!dw || !dwb || !dX || !dY || !didx || !dg || !dl) {
        g_create_error = "rb_mlp_grad: device allocation failed";
        return RB_ERR_CUDA;
    }
    std::vector<float> pad(np);
    mlp::to_padded(w, pad.data());
    std::vector<int32_t> idx(n);
    for (int64_t i = 0; i < n; i++) idx[i] = (int32_t)i;
    cudaMemcpyAsync(dw, pad.data(), sizeof(float) * np, cudaMemcpyHostToDevice, B.s);
    cudaMemcpyAsync(dX, X, sizeof(float) * 12 * n, cudaMemcpyHostToDevice, B.s);
    cudaMemcpyAsync(dY, Y, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, B.s);
    cudaMemcpyAsync(didx, idx.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, B.s);
    cudaMemsetAsync(dl, 0, sizeof(float), B.s);
    mlp::to_bf16_async(dw, dwb, B.s);
    if (mlp::grad_async(dwb, dw, dX, dY, didx, (int)n, (int)n, dg, dl, B.s) != cudaSuccess) {
        g_create_error = "rb_mlp_grad: launch failed";
        return RB_ERR_CUDA;
    }
    float lsum = 0.f;
    cudaMemcpyAsync(pad.data(), dg, sizeof(float) * np, cudaMemcpyDeviceToHost, B.s);
    cudaMemcpyAsync(&lsum, dl, sizeof(float), cudaMemcpyDeviceToHost, B.s);
    if (cudaStreamSynchronize(B.s) != cudaSuccess) {
        g_create_error = "rb_mlp_grad: CUDA error";
        return RB_ERR_CUDA;
    }
    mlp::from_padded(pad.data(), grad);
    if (loss) *loss = lsum / (3.0f * (float)n);
    return RB_OK;
}

int rb_mlp_grad_fp32(const float* w, const float* X, const float* Y, int64_t n, float* grad,
                     float* loss, void* cuda_stream) {
    if (!w || !X || !Y || n < 1 || n > 4096 || !grad) {
        g_create_error = "rb_mlp_grad_fp32: bad arguments (1 <= n <= 4096)";
        return RB_ERR_ARG;
    }
    MlpBufs B;
    B.s = static_cast<cudaStream_t>(cuda_stream);
    if (!B.s) {
        cudaStreamCreateWithFlags(&B.s, cudaStreamNonBlocking);
        B.own = true;
    }
    float* dw = B.alloc<float>(RB_MLP_PARAMS);
    float* dX = B.alloc<float>(12 * n);
    float* dY = B.alloc<float>(3 * n);
    float* dG = B.alloc<float>((size_t)n * RB_MLP_PARAMS);
    float* dl = B.alloc<float>(n);
    float* dg = B.alloc<float>(RB_MLP_PARAMS);
    float* dloss = B.alloc<float>(1);
    if (!dw || !dX || !dY || !dG || !dl || !dg || !dloss) {
        g_create_error = "rb_mlp_grad_fp32: device allocation failed";
        return RB_ERR_CUDA;
    }
    cudaMemcpyAsync(dw, w, sizeof(float) * RB_MLP_PARAMS, cudaMemcpyHostToDevice, B.s);
    cudaMemcpyAsync(dX, X, sizeof(float) * 12 * n, cudaMemcpyHostToDevice, B.s);
    cudaMemcpyAsync(dY, Y, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, B.s);
    if (mlp::grad_f32_async(dw, dX, dY, (int)n, dG, dl, dg, dloss, B.s) != cudaSuccess) {
        g_create_error = "rb_mlp_grad_fp32: launch failed";
        return RB_ERR_CUDA;
    }
    float lsum = 0.f;
    cudaMemcpyAsync(grad, dg, sizeof(float) * RB_MLP_PARAMS, cudaMemcpyDeviceToHost, B.s);
    cudaMemcpyAsync(&lsum, dloss, sizeof(float), cudaMemcpyDeviceToHost, B.s);
    if (cudaStreamSynchronize(B.s) != cudaSuccess) {
        g_create_error = "rb_mlp_grad_fp32: CUDA error";
        return RB_ERR_CUDA;
    }
    if (loss) *loss = lsum;
    return RB_OK;
}

int rb_mlp_train(const float* X, const float* Y, int64_t n, int epochs, int batch, double lr,
                 uint64_t seed, const float* w_init, float* w_out, float* loss_hist,
                 void* cuda_stream) {
    if (!X || !Y || n < 1 || n > 0x7fffffffll || epochs < 1 || batch < 16 || !(lr > 0.0) || !w_init ||
        !w_out) {
        g_create_error = "rb_mlp_train: bad arguments";
        return RB_ERR_ARG;
    }
    MlpBufs B;
    B.s = static_cast<cudaStream_t>(cuda_stream);
    if (!B.s) {
        cudaStreamCreateWithFlags(&B.s, cudaStreamNonBlocking);
        B.own = true;
    }
    const int np = mlp::padded_size();
    float* dw = B.alloc<float>(np);
    float* dm = B.alloc<float>(np);
    float* dv = B.alloc<float>(np);
    uint16_t* dwb = B.alloc<uint16_t>(np);
    float* dX = B.alloc<float>(12 * n);
    float* dY = B.alloc<float>(3 * n);
    int32_t* didx = B.alloc<int32_t>(n);
    float* dg = B.alloc<float>(np);
    float* dl = B.alloc<float>(epochs);
    if (!dw || !dm || !dv || !dwb || !dX || !dY || !didx || !dg || !dl) {
        g_create_error = "rb_mlp_train: device allocation failed";
        return RB_ERR_CUDA;
    }
    std::vector<float> pad(np);
    mlp::to_padded(w_init, pad.data());
    // train on standardised inputs and outputs (zero mean, unit variance per
    // column); the scales are folded back into W1, b1, W4, b4 at the end, so
    // w_init is in standardised units and w_out in raw units
    double mu[15] = {0}, sd[15] = {0};
    for (int64_t i = 0; i < n; i++) {
        for (int c = 0; c < 12; c++) mu[c] += X[i * 12 + c];
        for (int c = 0; c < 3; c++) mu[12 + c] += Y[i * 3 + c];
    }
    for (int c = 0; c < 15; c++) mu[c] /= (double)n;
    for (int64_t i = 0; i < n; i++) {
        for (int c = 0; c < 12; c++) sd[c] += (X[i * 12 + c] - mu[c]) * (X[i * 12 + c] - mu[c]);
        for (int c = 0; c < 3; c++) sd[12 + c] += (Y[i * 3 + c] - mu[12 + c]) * (Y[i * 3 + c] - mu[12 + c]);
    }
    for (int c = 0; c < 15; c++) sd[c] = sd[c] > 0.0 ? std::sqrt(sd[c] / (double)n) : 1.0;
    std::vector<float> Xn((size_t)n * 12), Yn((size_t)n * 3);
    for (int64_t i = 0; i < n; i++) {
        for (int c = 0; c < 12; c++) Xn[i * 12 + c] = (float)((X[i * 12 + c] - mu[c]) / sd[c]);
        for (int c = 0; c < 3; c++) Yn[i * 3 + c] = (float)((Y[i * 3 + c] - mu[12 + c]) / sd[12 + c]);
    }
    cudaMemcpyAsync(dw, pad.data(), sizeof(float) * np, cudaMemcpyHostToDevice, B.s);
    cudaMemsetAsync(dm, 0, sizeof(float) * np, B.s);
    cudaMemsetAsync(dv, 0, sizeof(float) * np, B.s);
    cudaMemsetAsync(dl, 0, sizeof(float) * epochs, B.s);
    cudaMemcpyAsync(dX, Xn.data(), sizeof(float) * 12 * n, cudaMemcpyHostToDevice, B.s);
    cudaMemcpyAsync(dY, Yn.data(), sizeof(float) * 3 * n, cudaMemcpyHostToDevice, B.s);
    mlp::to_bf16_async(dw, dwb, B.s);
    std::vector<int32_t> idx(n);
    std::mt19937_64 rng(seed);
    int step = 0;
    for (int ep = 0; ep < epochs; ep++) {
        for (int64_t i = 0; i < n; i++) idx[i] = (int32_t)i;
        std::shuffle(idx.begin(), idx.end(), rng);
        cudaMemcpyAsync(didx, idx.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, B.s);
        for (int64_t b0 = 0; b0 < n; b0 += batch) {
            const int nb = (int)std::min<int64_t>(batch, n - b0);
            if (mlp::grad_async(dwb, dw, dX, dY, didx + b0, nb, nb, dg, dl + ep, B.s) != cudaSuccess) {
                g_create_error = "rb_mlp_train: launch failed";
                return RB_ERR_CUDA;
            }
            mlp::adam_async(dw, dm, dv, dg, dwb, (float)lr, ++step, B.s);
        }
        // the host permutation buffer is reused next epoch
        if (cudaStreamSynchronize(B.s) != cudaSuccess) {
            g_create_error = "rb_mlp_train: CUDA error";
            return RB_ERR_CUDA;
        }
    }
    std::vector<float> losses(epochs);
    cudaMemcpyAsync(pad.data(), dw, sizeof(float) * np, cudaMemcpyDeviceToHost, B.s);
    cudaMemcpyAsync(losses.data(), dl, sizeof(float) * epochs, cudaMemcpyDeviceToHost, B.s);
    if (cudaStreamSynchronize(B.s) != cudaSuccess) {
        g_create_error = "rb_mlp_train: CUDA error";
        return RB_ERR_CUDA;
    }
    mlp::from_padded(pad.data(), w_out);
    // fold the standardisation into the weights: z1 = ((x - mu)/sd) W1 + b1 and
    // y = (h3 W4 + b4) sd_y + mu_y
    {
        float* W1 = w_out;              // 12 x 64
        float* b1 = w_out + 12 * 64;    // 64
        for (int o = 0; o < 64; o++) {
            double b = b1[o];
            for (int c = 0; c < 12; c++) {
                b -= mu[c] / sd[c] * W1[c * 64 + o];
                W1[c * 64 + o] = (float)(W1[c * 64 + o] / sd[c]);
            }
            b1[o] = (float)b;
        }
        float* W4 = w_out + RB_MLP_PARAMS - 3 - 64 * 3;   // 64 x 3
        float* b4 = w_out + RB_MLP_PARAMS - 3;
        for (int c = 0; c < 3; c++) {
            for (int h = 0; h < 64; h++) W4[h * 3 + c] = (float)(W4[h * 3 + c] * sd[12 + c]);
            b4[c] = (float)(b4[c] * sd[12 + c] + mu[12 + c]);
        }
    }
    // per-epoch mean loss in raw units (the standardised loss times the
    // mean output variance)
    const double var_y = (sd[12] * sd[12] + sd[13] * sd[13] + sd[14] * sd[14]) / 3.0;
    if (loss_hist)
        for (int ep = 0; ep < epochs; ep++)
            loss_hist[ep] = (float)(losses[ep] / (3.0 * (double)n) * var_y);
    return RB_OK;
}

int rb_sort_pairs_u64(int64_t n, int64_t cap, int key_bits, uint64_t* keys, uint32_t* vals,
                      void* cuda_stream) {
    if (n < 0 || cap < n || cap >= (int64_t(1) << 30) || key_bits < 1 || key_bits > 64 ||
        (n > 0 && !keys)) {
        set_global_error("rb_sort_pairs_u64: bad n, cap or key_bits, or keys missing");
        return RB_ERR_ARG;
    }
    if (cap == 0) return RB_OK;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int ncap = (int)cap;
    uint64_t *k0 = nullptr, *k1 = nullptr;
    uint32_t *v0 = nullptr, *v1 = nullptr, *hist = nullptr;
    int* dn = nullptr;   // [0]: count, [1]: error bits
    auto cleanup = [&]() {
        cudaFree(k0); cudaFree(k1); cudaFree(v0); cudaFree(v1); cudaFree(hist); cudaFree(dn);
    };
    auto cuda_fail = [&](cudaError_t e) {
        set_global_error(std::string("rb_sort_pairs_u64: ") + cudaGetErrorString(e));
        cleanup();
        return RB_ERR_CUDA;
    };
    cudaError_t e = cudaSuccess;
    if ((e = cudaMalloc(&k0, sizeof(uint64_t) * cap)) || (e = cudaMalloc(&k1, sizeof(uint64_t) * cap)) ||
        (e = cudaMalloc(&v0, sizeof(uint32_t) * cap)) || (e = cudaMalloc(&v1, sizeof(uint32_t) * cap)) ||
        (e = cudaMalloc(&hist, sizeof(uint32_t) * radix_hist_words(ncap))) ||
        (e = cudaMalloc(&dn, 2 * sizeof(int))))
        return cuda_fail(e);
    const int hn[2] = {(int)n, 0};
    if ((e = cudaMemcpyAsync(dn, hn, sizeof(hn), cudaMemcpyHostToDevice, st)) ||
        (n > 0 && (e = cudaMemcpyAsync(k0, keys, sizeof(uint64_t) * n, cudaMemcpyHostToDevice, st))))
        return cuda_fail(e);
    if (n > 0 && vals && (e = cudaMemcpyAsync(v0, vals, sizeof(uint32_t) * n, cudaMemcpyHostToDevice, st)))
        return cuda_fail(e);
    cudaGetLastError();
    const int which = radix_sort(k0, v0, k1, v1, ncap, dn, key_bits, nullptr, 0, hist, dn + 1, st);
    if ((e = cudaGetLastError())) return cuda_fail(e);
    int herr[2] = {0, 0};
    if ((e = cudaMemcpyAsync(herr, dn, sizeof(herr), cudaMemcpyDeviceToHost, st)) ||
        (n > 0 && (e = cudaMemcpyAsync(keys, which ? k1 : k0, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost, st))))
        return cuda_fail(e);
    if (n > 0 && vals &&
        (e = cudaMemcpyAsync(vals, which ? v1 : v0, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, st)))
        return cuda_fail(e);
    if ((e = cudaStreamSynchronize(st))) return cuda_fail(e);
    cleanup();
    if (herr[1] & kErrSortStall) {
        set_global_error("rb_sort_pairs_u64: a bounded look-back wait gave up");
        return RB_ERR_TIMEOUT;
    }
    return RB_OK;
}

}  // extern "C"
