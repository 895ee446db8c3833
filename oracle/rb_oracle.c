/*
 * rb_oracle.c -- plain, slow FP64 CPU oracle for the tree gravity and tree
 * collision hot path of REBOUND (Rein & Liu 2012).
 *
 * TEST INFRASTRUCTURE ONLY: it is loaded by the tests, by the smoke check and
 * by the bench's CPU-baseline leg, never by the product path.  It shares no
 * code, header or table with the CUDA library.  Compile with
 * -ffp-contract=off: every floating-point expression here is meant to be
 * evaluated exactly in the order written.
 *
 * Each function names the passage of the paper it follows.  Where the paper
 * is silent or garbled the reading taken is stated next to the code:
 *  R1  Eq. 1 prints a unit vector under a 3/2 power; the separation vector
 *      r_ji = x_j - x_i is used (Plummer softening b).
 *  R2  Sect. 4.2 insertion never stops for coincident particles; the depth is
 *      capped at 21 levels and a depth-21 cell holding several particles is a
 *      leaf group whose members are always interacted one by one.
 *  R3  Sect. 4.2 cites Hernquist (1987) for the quadrupole: the traceless
 *      Q_ab = sum m (3 d_a d_b - |d|^2 delta_ab) about the centre of mass.
 *  R4  Sect. 4.2 opening angle: a cell is used when w < theta R (strict),
 *      evaluated as w*w < (theta*theta)*R^2, and only when the target point
 *      is not inside the cell's closed cube.
 *  R5  softening applies to particle terms and to the monopole term only.
 *  R6  Sect. 2.3 gives no shear-offset formula: standard shearing-sheet
 *      images with offset (gx Lx, gy Ly - gx s, gz Lz), s = fmod(1.5 Omega
 *      Lx t, Ly), and velocity offset -1.5 Omega Lx gx in y.
 *  R7  Sect. 3.3 gives no SEI formula: the exact solution of Hill's
 *      equations without forces is the drift, the kick is v += a dt.
 *  R8  Sect. 5: collisions are found when particles overlap at the end of the
 *      step and resolved in ascending (id_a, id_b, image) order instead of a
 *      random shuffle, so that results are reproducible.
 *  S1  Sect. 5.3 approximates trajectories by straight lines between the
 *      positions before and after the drift: at detection time t (the end of
 *      the step) particle i moves on x_i + v_i tau, tau in [-dt/2, dt/2] (the
 *      merged drift around t, during which velocities do not change).
 *  S2  Sect. 5.3 does not define "a collision during the time-step": two
 *      lines collide when their smallest distance over that interval is below
 *      R_a + R_b (closest approach tau* = -(r.u)/|u|^2, clamped).
 *  S3  the x extent of a trajectory is [x - |v_x| dt/2 - R, x + |v_x| dt/2 + R]
 *      (both drift ends, widened by the radius), plus 1e-9 Lx on each side so
 *      rounding cannot drop a pair; ghost images in x are copies shifted by
 *      +k Lx that are only tested against original particles.
 *  S4  pairs from the sweep use the key and queue order of R8 and the same
 *      resolution (Eq. 2); a pair that is receding at t is not resolved.
 *  T1  Sect. 4 counts the particles that exert gravity separately from those
 *      that only feel it (N_active): particles with id >= n_active are test
 *      particles, their mass counts for collisions and kinetic energy but
 *      not as a source of Eq. 1 (the tree holds them with zero source mass).
 *  V1  Sect. 5 allows a velocity-dependent coefficient of restitution without
 *      fixing a law: law 1 is the power law eps = min(1, (|v_n|/v_c)^(-p))
 *      (|v_n| the normal approach speed), law 0 the constant eps.
 */
#include "rb_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

const char* orc_version(void) { return "rb_oracle 1"; }

int orc_nthreads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Boundaries and ghost images (Sect. 2.3, reading R6)                       */
/* ------------------------------------------------------------------------ */

/* Time after `half_step` drift halves: t0 + h * (dt / 2) (Sect. 3, DKD). */
double orc_time(const orc_params* p, int64_t half_step) {
    return p->t0 + (double)half_step * (0.5 * p->dt);
}

static double shear_speed(const orc_params* p) {
    if (p->boundary != ORC_BC_SHEAR) return 0.0;
    return (1.5 * p->omega) * p->L[0];
}

static double shear_offset(const orc_params* p, double t) {
    if (p->boundary != ORC_BC_SHEAR) return 0.0;
    return fmod(shear_speed(p) * t, p->L[1]);
}

/* The ghost boxes of Sect. 2.3: every (gx, gy, gz) in the cube of half-width
 * nghost; gx outermost.  Open boundaries have only the central image. */
int orc_images(const orc_params* p, double t, int cap, double* off, double* dvy, int* code) {
    int ng[3] = {p->nghost[0], p->nghost[1], p->nghost[2]};
    if (p->boundary == ORC_BC_OPEN) ng[0] = ng[1] = ng[2] = 0;
    if (!p->z_periodic) ng[2] = 0;
    double s = shear_offset(p, t), vs = shear_speed(p);
    int k = 0;
    for (int gx = -ng[0]; gx <= ng[0]; gx++)
        for (int gy = -ng[1]; gy <= ng[1]; gy++)
            for (int gz = -ng[2]; gz <= ng[2]; gz++) {
                if (k >= cap) return k;
                off[3 * k + 0] = (double)gx * p->L[0];
                off[3 * k + 1] = (double)gy * p->L[1] - (double)gx * s;
                off[3 * k + 2] = (double)gz * p->L[2];
                dvy[k] = -(double)gx * vs;
                code[k] = (gx + 7) | ((gy + 7) << 4) | ((gz + 7) << 8);
                k++;
            }
    return k;
}

#define ORC_CENTRAL_CODE (7 | (7 << 4) | (7 << 8))
#define ORC_MAXIMG 343

/* Boundary conditions after a drift half (Sect. 2.3): open boundaries remove
 * particles that left the root cube; periodic and shear-periodic ones wrap
 * them (reading R6).  Removal keeps the survivors in their order.  Returns
 * the new particle count. */
int64_t orc_boundary(const orc_params* p, double t, int64_t n, double* x, double* y, double* z,
                     double* vx, double* vy, double* vz, double* m, double* r, int64_t* id) {
    double Lx = p->L[0], Ly = p->L[1], Lz = p->L[2];
    double hx = 0.5 * Lx, hy = 0.5 * Ly, hz = 0.5 * Lz;
    double s = shear_offset(p, t), vs = shear_speed(p);
    int64_t w = 0;
    for (int64_t i = 0; i < n; i++) {
        int keep = 1;
        if (p->boundary == ORC_BC_OPEN) {
            if (x[i] < -hx || x[i] >= hx || y[i] < -hy || y[i] >= hy || z[i] < -hz || z[i] >= hz)
                keep = 0;
        } else {
            if (x[i] >= hx) {
                x[i] = x[i] - Lx;
                y[i] = y[i] + s;
                vy[i] = vy[i] + vs;
            } else if (x[i] < -hx) {
                x[i] = x[i] + Lx;
                y[i] = y[i] - s;
                vy[i] = vy[i] - vs;
            }
            while (y[i] >= hy) y[i] = y[i] - Ly;
            while (y[i] < -hy) y[i] = y[i] + Ly;
            if (p->z_periodic) {
                while (z[i] >= hz) z[i] = z[i] - Lz;
                while (z[i] < -hz) z[i] = z[i] + Lz;
            } else if (z[i] < -hz || z[i] >= hz) {
                keep = 0;
            }
        }
        if (keep) {
            x[w] = x[i]; y[w] = y[i]; z[w] = z[i];
            vx[w] = vx[i]; vy[w] = vy[i]; vz[w] = vz[i];
            m[w] = m[i]; r[w] = r[i]; id[w] = id[i];
            w++;
        }
    }
    return w;
}

/* ------------------------------------------------------------------------ */
/* Integrators (Sect. 3)                                                     */
/* ------------------------------------------------------------------------ */

/* Drift for dt/2.  Leap-frog (Sect. 3.1): x += v dt/2.  SEI (Sect. 3.3,
 * reading R7): the exact solution of Hill's equations
 *   x'' - 2 Omega y' - 3 Omega^2 x = 0,  y'' + 2 Omega x' = 0,
 *   z'' + Omega_z^2 z = 0
 * over tau = dt/2. */
void orc_drift(const orc_params* p, int64_t n, double* x, double* y, double* z, double* vx,
               double* vy, double* vz) {
    double tau = 0.5 * p->dt;
    if (p->integrator == ORC_INT_LEAPFROG) {
        for (int64_t i = 0; i < n; i++) {
            x[i] = x[i] + vx[i] * tau;
            y[i] = y[i] + vy[i] * tau;
            z[i] = z[i] + vz[i] * tau;
        }
        return;
    }
    double O = p->omega, Oz = p->omega_z > 0.0 ? p->omega_z : p->omega;
    double ph = O * tau, c = cos(ph), s = sin(ph);
    double phz = Oz * tau, cz = cos(phz), sz = sin(phz);
    /* coefficients of the linear map (x, vx, vy) -> (x, y, vx, vy) */
    double axx = 4.0 - 3.0 * c, axu = s / O, axv = (2.0 / O) * (1.0 - c);
    double ayx = 6.0 * (s - ph), ayu = -(2.0 / O) * (1.0 - c), ayv = (4.0 * s - 3.0 * ph) / O;
    double aux = (3.0 * O) * s, auu = c, auv = 2.0 * s;
    double avx = (6.0 * O) * (c - 1.0), avu = -2.0 * s, avv = 4.0 * c - 3.0;
    double azz = cz, azw = sz / Oz, awz = -(Oz * sz), aww = cz;
    for (int64_t i = 0; i < n; i++) {
        double x0 = x[i], u0 = vx[i], v0 = vy[i], z0 = z[i], w0 = vz[i];
        x[i] = (axx * x0 + axu * u0) + axv * v0;
        y[i] = y[i] + ((ayx * x0 + ayu * u0) + ayv * v0);
        vx[i] = (aux * x0 + auu * u0) + auv * v0;
        vy[i] = (avx * x0 + avu * u0) + avv * v0;
        z[i] = azz * z0 + azw * w0;
        vz[i] = awz * z0 + aww * w0;
    }
}

/* Kick for a full dt (Sect. 3, DKD): v += a dt.  For SEI the acceleration
 * holds only the non-epicyclic forces (self-gravity). */
void orc_kick(const orc_params* p, int64_t n, double* vx, double* vy, double* vz,
              const double* ax, const double* ay, const double* az) {
    for (int64_t i = 0; i < n; i++) {
        vx[i] = vx[i] + ax[i] * p->dt;
        vy[i] = vy[i] + ay[i] * p->dt;
        vz[i] = vz[i] + az[i] * p->dt;
    }
}

/* ------------------------------------------------------------------------ */
/* Direct summation (Sect. 4, Eq. 1, reading R1; Sect. 4.1)                  */
/* ------------------------------------------------------------------------ */

/* a_i = sum over images g and particles j (except j = i in the central
 * image) of G m_j (x_j + off_g - x_i) / (|x_j + off_g - x_i|^2 + b^2)^(3/2).
 * The potential phi_i = -sum G m_j / sqrt(|.|^2 + b^2) is returned too.
 * Only the targets listed in tsel are computed (all when tsel == NULL). */
void orc_direct_gravity(const orc_params* p, double t, int64_t n, const double* x, const double* y,
                        const double* z, const double* m, int64_t nt, const int64_t* tsel,
                        double* ax, double* ay, double* az, double* phi) {
    double off[3 * ORC_MAXIMG], dvy[ORC_MAXIMG];
    int code[ORC_MAXIMG];
    int ni = orc_images(p, t, ORC_MAXIMG, off, dvy, code);
    double b2 = p->soft * p->soft, G = p->G;
    int64_t cnt = tsel ? nt : n;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < cnt; k++) {
        int64_t i = tsel ? tsel[k] : k;
        double sx = 0.0, sy = 0.0, sz = 0.0, sp = 0.0;
        for (int g = 0; g < ni; g++) {
            /* the target point seen from the sources of image g */
            double px = x[i] - off[3 * g + 0];
            double py = y[i] - off[3 * g + 1];
            double pz = z[i] - off[3 * g + 2];
            for (int64_t j = 0; j < n; j++) {
                if (j == i && code[g] == ORC_CENTRAL_CODE) continue;
                double dx = x[j] - px, dy = y[j] - py, dz = z[j] - pz;
                double r2 = ((dx * dx + dy * dy) + dz * dz) + b2;
                double inv = 1.0 / sqrt(r2);
                double f = G * m[j] * (inv * inv * inv);
                sx = sx + f * dx;
                sy = sy + f * dy;
                sz = sz + f * dz;
                sp = sp - G * m[j] * inv;
            }
        }
        ax[k] = sx; ay[k] = sy; az[k] = sz;
        if (phi) phi[k] = sp;
    }
}

/* ------------------------------------------------------------------------ */
/* Octree by insertion (Sect. 4.2, readings R2-R4)                           */
/* ------------------------------------------------------------------------ */

typedef struct {
    int child[8];       /* -1: no child in this octant */
    int depth;          /* root = 0; width = L / 2^depth */
    int64_t ix, iy, iz; /* integer index of the cell at its depth */
    int64_t npart;      /* particles in the subtree */
    int64_t leafp;      /* the particle of a one-particle leaf, else -1 */
    int64_t* group;     /* members of a depth-21 leaf group */
    int64_t ngroup, capgroup;
    double M, com[3], Q[6]; /* Q order: xx, yy, zz, xy, xz, yz */
} orc_node;

struct orc_tree {
    orc_node* nodes;
    int64_t nnodes, capnodes;
    int64_t n;
    const double *x, *y, *z, *m;
    double L, lo;
    int64_t* kx; /* integer coordinates of every particle */
    int64_t* ky;
    int64_t* kz;
};

/* Integer coordinate of a position: floor(((x - lo) / L) * 2^21), clamped. */
static int64_t orc_icoord(double x, double lo, double L) {
    double u = (x - lo) / L;
    double k = floor(u * 2097152.0);
    if (!(k >= 0.0)) k = 0.0;
    if (k > 2097151.0) k = 2097151.0;
    return (int64_t)k;
}

static int orc_octant(const orc_tree* t, int64_t q, int depth) {
    int sh = 20 - depth;
    int bx = (int)((t->kx[q] >> sh) & 1), by = (int)((t->ky[q] >> sh) & 1);
    int bz = (int)((t->kz[q] >> sh) & 1);
    return (bx << 2) | (by << 1) | bz;
}

static int orc_new_child(orc_tree* t, int parent, int oct) {
    if (t->nnodes == t->capnodes) {
        t->capnodes = t->capnodes ? 2 * t->capnodes : 1024;
        t->nodes = (orc_node*)realloc(t->nodes, (size_t)t->capnodes * sizeof(orc_node));
    }
    int c = (int)t->nnodes++;
    orc_node* nd = &t->nodes[c];
    memset(nd, 0, sizeof(*nd));
    for (int o = 0; o < 8; o++) nd->child[o] = -1;
    nd->leafp = -1;
    if (parent >= 0) {
        orc_node* pa = &t->nodes[parent];
        nd->depth = pa->depth + 1;
        nd->ix = 2 * pa->ix + ((oct >> 2) & 1);
        nd->iy = 2 * pa->iy + ((oct >> 1) & 1);
        nd->iz = 2 * pa->iz + (oct & 1);
        pa->child[oct] = c;
    }
    return c;
}

static void orc_group_push(orc_node* nd, int64_t q) {
    if (nd->ngroup == nd->capgroup) {
        nd->capgroup = nd->capgroup ? 2 * nd->capgroup : 4;
        nd->group = (int64_t*)realloc(nd->group, (size_t)nd->capgroup * sizeof(int64_t));
    }
    nd->group[nd->ngroup++] = q;
}

/* Add one particle: descend to an empty leaf; split an occupied one-particle
 * leaf into eight octants (Sect. 4.2); at the depth cap, grow the group. */
static void orc_insert(orc_tree* t, int64_t q) {
    int nd = 0;
    for (;;) {
        orc_node* c = &t->nodes[nd];
        if (c->npart == 0) {
            c->leafp = q;
            c->npart = 1;
            return;
        }
        if (c->depth == ORC_MAXDEPTH) {
            if (c->ngroup == 0) orc_group_push(c, c->leafp);
            c->leafp = -1;
            orc_group_push(c, q);
            c->npart++;
            return;
        }
        if (c->npart == 1) {
            int64_t old = c->leafp;
            c->leafp = -1;
            int o = orc_octant(t, old, c->depth);
            int k = orc_new_child(t, nd, o);
            t->nodes[k].leafp = old;
            t->nodes[k].npart = 1;
        }
        c = &t->nodes[nd];
        c->npart++;
        int o = orc_octant(t, q, c->depth);
        if (c->child[o] < 0) orc_new_child(t, nd, o);
        nd = t->nodes[nd].child[o];
    }
}

/* Append the particles of a subtree to out (returns the new length). */
static int64_t orc_collect(const orc_tree* t, int nd, int64_t* out, int64_t k) {
    const orc_node* c = &t->nodes[nd];
    if (c->leafp >= 0) {
        out[k++] = c->leafp;
        return k;
    }
    if (c->ngroup > 0) {
        for (int64_t g = 0; g < c->ngroup; g++) out[k++] = c->group[g];
        return k;
    }
    for (int o = 0; o < 8; o++)
        if (c->child[o] >= 0) k = orc_collect(t, c->child[o], out, k);
    return k;
}

/* Cell moments straight from their definitions over the cell's particles
 * (Sect. 4.2: mass and centre of mass; reading R3 for the quadrupole).  A
 * massless cell takes its geometric centre as centre of mass. */
static void orc_moments(orc_tree* t, int64_t* scratch) {
    for (int64_t c = 0; c < t->nnodes; c++) {
        orc_node* nd = &t->nodes[c];
        int64_t k = orc_collect(t, (int)c, scratch, 0);
        double M = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
        for (int64_t a = 0; a < k; a++) {
            int64_t q = scratch[a];
            M = M + t->m[q];
            sx = sx + t->m[q] * t->x[q];
            sy = sy + t->m[q] * t->y[q];
            sz = sz + t->m[q] * t->z[q];
        }
        double w = ldexp(t->L, -nd->depth);
        if (M > 0.0) {
            nd->com[0] = sx / M; nd->com[1] = sy / M; nd->com[2] = sz / M;
        } else {
            nd->com[0] = t->lo + ((double)nd->ix + 0.5) * w;
            nd->com[1] = t->lo + ((double)nd->iy + 0.5) * w;
            nd->com[2] = t->lo + ((double)nd->iz + 0.5) * w;
        }
        double Q[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t a = 0; a < k; a++) {
            int64_t q = scratch[a];
            double dx = t->x[q] - nd->com[0], dy = t->y[q] - nd->com[1];
            double dz = t->z[q] - nd->com[2];
            double d2 = (dx * dx + dy * dy) + dz * dz, mq = t->m[q];
            Q[0] = Q[0] + mq * (3.0 * dx * dx - d2);
            Q[1] = Q[1] + mq * (3.0 * dy * dy - d2);
            Q[2] = Q[2] + mq * (3.0 * dz * dz - d2);
            Q[3] = Q[3] + mq * (3.0 * dx * dy);
            Q[4] = Q[4] + mq * (3.0 * dx * dz);
            Q[5] = Q[5] + mq * (3.0 * dy * dz);
        }
        nd->M = M;
        memcpy(nd->Q, Q, sizeof(Q));
    }
}

/* Build the tree of Sect. 4.2 over the root cube [-L/2, L/2)^3 by inserting
 * the particles one at a time in index order, then compute the moments. */
orc_tree* orc_tree_build(int64_t n, const double* x, const double* y, const double* z,
                         const double* m, double L) {
    orc_tree* t = (orc_tree*)calloc(1, sizeof(orc_tree));
    t->n = n; t->x = x; t->y = y; t->z = z; t->m = m;
    t->L = L; t->lo = -0.5 * L;
    t->kx = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    t->ky = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    t->kz = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    for (int64_t q = 0; q < n; q++) {
        t->kx[q] = orc_icoord(x[q], t->lo, L);
        t->ky[q] = orc_icoord(y[q], t->lo, L);
        t->kz[q] = orc_icoord(z[q], t->lo, L);
    }
    orc_new_child(t, -1, 0); /* root */
    for (int64_t q = 0; q < n; q++) orc_insert(t, q);
    int64_t* scratch = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    orc_moments(t, scratch);
    free(scratch);
    return t;
}

void orc_tree_free(orc_tree* t) {
    if (!t) return;
    for (int64_t c = 0; c < t->nnodes; c++) free(t->nodes[c].group);
    free(t->nodes); free(t->kx); free(t->ky); free(t->kz);
    free(t);
}

/* A cell is "canonical" when it is a leaf group or has two or more non-empty
 * octants; cells with a single non-empty octant hold the same particle set as
 * that octant and are left out (the forces do not depend on them). */
static int orc_canonical(const orc_node* nd) {
    if (nd->ngroup > 0) return 1;
    if (nd->leafp >= 0 || nd->npart < 2) return 0;
    int k = 0;
    for (int o = 0; o < 8; o++) k += nd->child[o] >= 0;
    return k >= 2;
}

int64_t orc_tree_ncells(const orc_tree* t) {
    int64_t k = 0;
    for (int64_t c = 0; c < t->nnodes; c++) k += orc_canonical(&t->nodes[c]);
    return k;
}

/* Canonical cells with their depth, particle count, members (concatenated
 * particle indices) and moments.  Returns the number of cells written. */
int64_t orc_tree_cells(const orc_tree* t, int64_t cap, int* depth, int64_t* count, int64_t* members,
                       int64_t members_cap, double* M, double* com, double* Q) {
    int64_t k = 0, mk = 0;
    for (int64_t c = 0; c < t->nnodes && k < cap; c++) {
        const orc_node* nd = &t->nodes[c];
        if (!orc_canonical(nd)) continue;
        depth[k] = nd->depth;
        count[k] = nd->npart;
        if (members && mk + nd->npart <= members_cap) mk = orc_collect(t, (int)c, members, mk);
        if (M) M[k] = nd->M;
        if (com) memcpy(com + 3 * k, nd->com, 3 * sizeof(double));
        if (Q) memcpy(Q + 6 * k, nd->Q, 6 * sizeof(double));
        k++;
    }
    return k;
}

typedef struct {
    double ax, ay, az, phi;
    int64_t ncell, nleaf, nmac;
} orc_acc;

/* Exact particle term of Eq. 1 (reading R1): source j at x_j, target point p. */
static void orc_pp(const orc_tree* t, const orc_params* p, int64_t j, const double* pt, orc_acc* a) {
    double dx = t->x[j] - pt[0], dy = t->y[j] - pt[1], dz = t->z[j] - pt[2];
    double r2 = ((dx * dx + dy * dy) + dz * dz) + p->soft * p->soft;
    double inv = 1.0 / sqrt(r2);
    double f = p->G * t->m[j] * (inv * inv * inv);
    a->ax = a->ax + f * dx;
    a->ay = a->ay + f * dy;
    a->az = a->az + f * dz;
    a->phi = a->phi - p->G * t->m[j] * inv;
    a->nleaf++;
}

/* Multipole term of an accepted cell (Sect. 4.2; readings R3, R5).  With
 * r = p - COM:  phi = -G M / |r| - G (r.Q.r) / (2 |r|^5),
 *   a = -G M r / |r|^3 + G [ Q r / |r|^5 - (5/2) (r.Q.r) r / |r|^7 ].
 * Here d = COM - p = -r is used. */
static void orc_cell(const orc_params* p, const orc_node* nd, const double* pt, orc_acc* a) {
    double dx = nd->com[0] - pt[0], dy = nd->com[1] - pt[1], dz = nd->com[2] - pt[2];
    double r2 = (dx * dx + dy * dy) + dz * dz;
    double rs2 = r2 + p->soft * p->soft;
    double invs = 1.0 / sqrt(rs2);
    double f = p->G * nd->M * (invs * invs * invs);
    a->ax = a->ax + f * dx;
    a->ay = a->ay + f * dy;
    a->az = a->az + f * dz;
    a->phi = a->phi - p->G * nd->M * invs;
    if (p->quadrupole) {
        const double* Q = nd->Q;
        double inv = 1.0 / sqrt(r2);
        double inv2 = inv * inv;
        double inv5 = inv2 * inv2 * inv;
        double inv7 = inv5 * inv2;
        double qx = (Q[0] * dx + Q[3] * dy) + Q[4] * dz;
        double qy = (Q[3] * dx + Q[1] * dy) + Q[5] * dz;
        double qz = (Q[4] * dx + Q[5] * dy) + Q[2] * dz;
        double dqd = (dx * qx + dy * qy) + dz * qz;
        double c = 2.5 * dqd * inv7;
        a->ax = a->ax + p->G * (c * dx - qx * inv5);
        a->ay = a->ay + p->G * (c * dy - qy * inv5);
        a->az = a->az + p->G * (c * dz - qz * inv5);
        a->phi = a->phi - p->G * (0.5 * dqd * inv5);
    }
    a->ncell++;
}

/* Opening-angle test (Sect. 4.2, reading R4). */
static int orc_accept(const orc_tree* t, const orc_params* p, const orc_node* nd, const double* pt) {
    double w = ldexp(t->L, -nd->depth);
    double dx = nd->com[0] - pt[0], dy = nd->com[1] - pt[1], dz = nd->com[2] - pt[2];
    double r2 = (dx * dx + dy * dy) + dz * dz;
    if (!(w * w < (p->theta * p->theta) * r2)) return 0;
    double cx = t->lo + (double)nd->ix * w, cy = t->lo + (double)nd->iy * w;
    double cz = t->lo + (double)nd->iz * w;
    int inside = cx <= pt[0] && pt[0] <= cx + w && cy <= pt[1] && pt[1] <= cy + w && cz <= pt[2] &&
                 pt[2] <= cz + w;
    return !inside;
}

/* Barnes-Hut descent from cell nd for target point pt; `self` is the target
 * particle in the central image (excluded), -1 in the other images. */
static void orc_walk(const orc_tree* t, const orc_params* p, int nd, const double* pt, int64_t self,
                     orc_acc* a) {
    const orc_node* c = &t->nodes[nd];
    if (c->npart == 0) return;
    if (c->leafp >= 0) {
        if (c->leafp != self) orc_pp(t, p, c->leafp, pt, a);
        return;
    }
    if (c->ngroup > 0) {
        for (int64_t g = 0; g < c->ngroup; g++)
            if (c->group[g] != self) orc_pp(t, p, c->group[g], pt, a);
        return;
    }
    a->nmac++;
    if (orc_accept(t, p, c, pt)) {
        orc_cell(p, c, pt, a);
        return;
    }
    for (int o = 0; o < 8; o++)
        if (c->child[o] >= 0) orc_walk(t, p, c->child[o], pt, self, a);
}

/* Tree gravity (Sect. 4.2) on the listed targets (all when tsel == NULL):
 * the tree is walked once per ghost image with the target point shifted by
 * minus the image offset.  Counts of accepted cells, exact particle terms
 * and opening tests are returned per target when the arrays are given. */
void orc_tree_gravity(const orc_tree* t, const orc_params* p, double t_now, int64_t nt,
                      const int64_t* tsel, double* ax, double* ay, double* az, double* phi,
                      int64_t* ncell, int64_t* nleaf, int64_t* nmac) {
    double off[3 * ORC_MAXIMG], dvy[ORC_MAXIMG];
    int code[ORC_MAXIMG];
    int ni = orc_images(p, t_now, ORC_MAXIMG, off, dvy, code);
    int64_t cnt = tsel ? nt : t->n;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < cnt; k++) {
        int64_t i = tsel ? tsel[k] : k;
        orc_acc a = {0, 0, 0, 0, 0, 0, 0};
        for (int g = 0; g < ni; g++) {
            double pt[3] = {t->x[i] - off[3 * g + 0], t->y[i] - off[3 * g + 1],
                            t->z[i] - off[3 * g + 2]};
            if (t->n > 0) orc_walk(t, p, 0, pt, code[g] == ORC_CENTRAL_CODE ? i : -1, &a);
        }
        ax[k] = a.ax; ay[k] = a.ay; az[k] = a.az;
        if (phi) phi[k] = a.phi;
        if (ncell) ncell[k] = a.ncell;
        if (nleaf) nleaf[k] = a.nleaf;
        if (nmac) nmac[k] = a.nmac;
    }
}

/* ------------------------------------------------------------------------ */
/* Collisions (Sect. 5, Eq. 2, Eq. 3; reading R8)                            */
/* ------------------------------------------------------------------------ */

static uint64_t orc_pair_key(int64_t a, int64_t b, int code) {
    return ((uint64_t)a << 36) | ((uint64_t)b << 12) | (uint64_t)code;
}

/* Overlap of particle b's image (offset o) with particle a (Sect. 5.1). */
static int orc_overlap(double xa, double ya, double za, double ra, double xb, double yb, double zb,
                       double rb, const double* o) {
    double rx = (xb + o[0]) - xa, ry = (yb + o[1]) - ya, rz = (zb + o[2]) - za;
    double r2 = (rx * rx + ry * ry) + rz * rz;
    double s = ra + rb;
    return r2 < s * s;
}

static int orc_cmp_u64(const void* a, const void* b) {
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* Direct nearest-neighbour search (Sect. 5.1): every pair of particles and
 * every image is tested once.  Returns the number of pairs (the first `cap`
 * are stored, sorted). */
int64_t orc_collide_brute(const orc_params* p, double t, int64_t n, const double* x, const double* y,
                          const double* z, const double* r, const int64_t* id, int64_t cap,
                          uint64_t* keys) {
    double off[3 * ORC_MAXIMG], dvy[ORC_MAXIMG];
    int code[ORC_MAXIMG];
    int ni = orc_images(p, t, ORC_MAXIMG, off, dvy, code);
    int64_t k = 0;
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = 0; j < n; j++) {
            if (id[i] >= id[j]) continue; /* a = lower id, b = higher id */
            for (int g = 0; g < ni; g++)
                if (orc_overlap(x[i], y[i], z[i], r[i], x[j], y[j], z[j], r[j], off + 3 * g)) {
                    if (k < cap) keys[k] = orc_pair_key(id[i], id[j], code[g]);
                    k++;
                }
        }
    qsort(keys, (size_t)(k < cap ? k : cap), sizeof(uint64_t), orc_cmp_u64);
    return k;
}

typedef struct {
    uint64_t* keys;
    int64_t k, cap;
} orc_pairbuf;

/* Eq. 3 descent: open cell c while r_ic < R_i + R_max + (sqrt(3)/2) w_c,
 * r_ic being the distance from the target point to the cell's centre. */
static void orc_csearch(const orc_tree* t, int nd, const double* pt, int64_t i, double ri,
                        double rmax, const double* r, const int64_t* id, const double* o, int code,
                        orc_pairbuf* pb) {
    const orc_node* c = &t->nodes[nd];
    if (c->npart == 0) return;
    int64_t single[1];
    const int64_t* mem = NULL;
    int64_t nm = 0;
    if (c->leafp >= 0) {
        single[0] = c->leafp;
        mem = single;
        nm = 1;
    } else if (c->ngroup > 0) {
        mem = c->group;
        nm = c->ngroup;
    }
    if (mem) {
        for (int64_t a = 0; a < nm; a++) {
            int64_t j = mem[a];
            if (j == i || id[i] >= id[j]) continue;
            if (orc_overlap(t->x[i], t->y[i], t->z[i], ri, t->x[j], t->y[j], t->z[j], r[j], o)) {
                if (pb->k < pb->cap) pb->keys[pb->k] = orc_pair_key(id[i], id[j], code);
                pb->k++;
            }
        }
        return;
    }
    double w = ldexp(t->L, -c->depth);
    double cx = t->lo + ((double)c->ix + 0.5) * w, cy = t->lo + ((double)c->iy + 0.5) * w;
    double cz = t->lo + ((double)c->iz + 0.5) * w;
    double dx = cx - pt[0], dy = cy - pt[1], dz = cz - pt[2];
    double ric = sqrt((dx * dx + dy * dy) + dz * dz);
    if (!(ric < ri + rmax + 0.5 * sqrt(3.0) * w)) return;
    for (int o8 = 0; o8 < 8; o8++)
        if (c->child[o8] >= 0) orc_csearch(t, c->child[o8], pt, i, ri, rmax, r, id, o, code, pb);
}

/* Tree nearest-neighbour search (Sect. 5.2, Eq. 3) on a tree built over the
 * given positions.  Every particle searches every image; a pair is recorded
 * by its lower-id member only, so each overlap is found once. */
int64_t orc_collide_tree(const orc_params* p, double t, int64_t n, const double* x, const double* y,
                         const double* z, const double* r, const int64_t* id, int64_t cap,
                         uint64_t* keys) {
    double off[3 * ORC_MAXIMG], dvy[ORC_MAXIMG];
    int code[ORC_MAXIMG];
    int ni = orc_images(p, t, ORC_MAXIMG, off, dvy, code);
    double* m1 = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    for (int64_t i = 0; i < n; i++) m1[i] = 1.0;
    orc_tree* tr = orc_tree_build(n, x, y, z, m1, p->L[0]);
    double rmax = 0.0;
    for (int64_t i = 0; i < n; i++) rmax = r[i] > rmax ? r[i] : rmax;
    orc_pairbuf pb = {keys, 0, cap};
    for (int64_t i = 0; i < n; i++)
        for (int g = 0; g < ni; g++) {
            /* the image of j at x_j + o is near x_i iff x_j is near x_i - o */
            double pt[3] = {x[i] - off[3 * g + 0], y[i] - off[3 * g + 1], z[i] - off[3 * g + 2]};
            if (n > 0) orc_csearch(tr, 0, pt, i, r[i], rmax, r, id, off + 3 * g, code[g], &pb);
        }
    orc_tree_free(tr);
    free(m1);
    qsort(keys, (size_t)(pb.k < cap ? pb.k : cap), sizeof(uint64_t), orc_cmp_u64);
    return pb.k;
}

/* The same Eq. 3 search run only from the listed targets (pairs that one of
 * them records as the lower-id member); used to time the search on a
 * sample.  Returns the number of pairs found (first `cap` stored, unsorted). */
/* Sect. 5.2 search from the listed targets on a tree already built over the
 * same positions (Eq. 3 uses only the cells' geometry, so a tree built with
 * any masses serves). */
int64_t orc_tree_collide_sel(const orc_tree* tr, const orc_params* p, double t, int64_t n,
                             const double* x, const double* y, const double* z, const double* r,
                             const int64_t* id, int64_t nt, const int64_t* tsel, int64_t cap,
                             uint64_t* keys) {
    double off[3 * ORC_MAXIMG], dvy[ORC_MAXIMG];
    int code[ORC_MAXIMG];
    int ni = orc_images(p, t, ORC_MAXIMG, off, dvy, code);
    double rmax = 0.0;
    for (int64_t i = 0; i < n; i++) rmax = r[i] > rmax ? r[i] : rmax;
    orc_pairbuf pb = {keys, 0, cap};
    for (int64_t k = 0; k < nt; k++) {
        int64_t i = tsel[k];
        for (int g = 0; g < ni; g++) {
            double pt[3] = {x[i] - off[3 * g + 0], y[i] - off[3 * g + 1], z[i] - off[3 * g + 2]};
            if (n > 0) orc_csearch(tr, 0, pt, i, r[i], rmax, r, id, off + 3 * g, code[g], &pb);
        }
    }
    return pb.k;
}

int64_t orc_collide_tree_sel(const orc_params* p, double t, int64_t n, const double* x,
                             const double* y, const double* z, const double* r, const int64_t* id,
                             int64_t nt, const int64_t* tsel, int64_t cap, uint64_t* keys) {
    double* m1 = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    for (int64_t i = 0; i < n; i++) m1[i] = 1.0;
    orc_tree* tr = orc_tree_build(n, x, y, z, m1, p->L[0]);
    int64_t k = orc_tree_collide_sel(tr, p, t, n, x, y, z, r, id, nt, tsel, cap, keys);
    orc_tree_free(tr);
    free(m1);
    return k;
}

/* ------------------------------------------------------------------------ */
/* Plane-sweep detection (Sect. 5.3; readings S1-S4)                         */
/* ------------------------------------------------------------------------ */

/* Straight-line criterion (reading S1): over the drift around the detection
 * time t each particle moves on x + v tau, tau in [-dt/2, dt/2] (the
 * positions before and after that drift are its ends).  Particle a and the
 * image of b (offset o, velocity offset dvy in y) collide when the smallest
 * distance between the two lines over that interval is below R_a + R_b. */
static int orc_line_hit(const orc_params* p, int64_t a, int64_t b, const double* x,
                        const double* y, const double* z, const double* vx, const double* vy,
                        const double* vz, const double* r, const double* o, double dvy) {
    double h = 0.5 * p->dt;
    double rx = (x[b] + o[0]) - x[a], ry = (y[b] + o[1]) - y[a], rz = (z[b] + o[2]) - z[a];
    double ux = vx[b] - vx[a], uy = (vy[b] + dvy) - vy[a], uz = vz[b] - vz[a];
    double uu = (ux * ux + uy * uy) + uz * uz;
    double ru = (rx * ux + ry * uy) + rz * uz;
    double tau = 0.0;
    if (uu > 0.0) {
        tau = -ru / uu; /* time of closest approach, clamped to the interval */
        if (tau < -h) tau = -h;
        if (tau > h) tau = h;
    }
    double dx = rx + ux * tau, dy = ry + uy * tau, dz = rz + uz * tau;
    double d2 = (dx * dx + dy * dy) + dz * dz;
    double s = r[a] + r[b];
    return d2 < s * s;
}

/* The straight-line criterion by brute force: every pair, every image. */
int64_t orc_collide_line_brute(const orc_params* p, double t, int64_t n, const double* x,
                               const double* y, const double* z, const double* vx, const double* vy,
                               const double* vz, const double* r, const int64_t* id, int64_t cap,
                               uint64_t* keys) {
    double off[3 * ORC_MAXIMG], dvy[ORC_MAXIMG];
    int code[ORC_MAXIMG];
    int ni = orc_images(p, t, ORC_MAXIMG, off, dvy, code);
    int64_t k = 0;
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = 0; j < n; j++) {
            if (id[i] >= id[j]) continue;
            for (int g = 0; g < ni; g++)
                if (orc_line_hit(p, i, j, x, y, z, vx, vy, vz, r, off + 3 * g, dvy[g])) {
                    if (k < cap) keys[k] = orc_pair_key(id[i], id[j], code[g]);
                    k++;
                }
        }
    qsort(keys, (size_t)(k < cap ? k : cap), sizeof(uint64_t), orc_cmp_u64);
    return k;
}

/* One stop of the plane: the x extent of an item's trajectory.  An item is a
 * particle (copy 0) or its copy shifted by +copy Lx (reading S3). */
typedef struct {
    double xs;
    int64_t item;
    int end; /* 0: the plane reaches the item (insert), 1: it leaves (remove) */
} orc_stop;

static int orc_cmp_stop(const void* a, const void* b) {
    const orc_stop *p = (const orc_stop*)a, *q = (const orc_stop*)b;
    if (p->xs != q->xs) return p->xs < q->xs ? -1 : 1;
    if (p->end != q->end) return p->end - q->end; /* inserts before removals */
    return p->item < q->item ? -1 : (p->item > q->item ? 1 : 0);
}

/* Plane sweep along x (Sect. 5.3).  Each trajectory's x extent (both ends of
 * the drift, widened by the radius; reading S3) gives two stops; the stops are
 * sorted; the plane visits them in order keeping the list of trajectories it
 * cuts (SWEEPL); a trajectory entering the list is tested against every
 * trajectory already in it with the straight-line criterion.  Ghost images
 * in x are copies of the particles shifted by +k Lx, k = 1..nghost[0]; a copy
 * is only tested against original particles, and every (pair, image) is
 * written in the canonical orientation (lower id a, image of b as seen from
 * a; reading S4).  Returns the number of pairs (first `cap` stored, sorted). */
int64_t orc_collide_sweep(const orc_params* p, double t, int64_t n, const double* x,
                          const double* y, const double* z, const double* vx, const double* vy,
                          const double* vz, const double* r, const int64_t* id, int64_t cap,
                          uint64_t* keys) {
    int ngx = p->boundary == ORC_BC_OPEN ? 0 : p->nghost[0];
    int ngy = p->boundary == ORC_BC_OPEN ? 0 : p->nghost[1];
    int ngz = (p->boundary == ORC_BC_OPEN || !p->z_periodic) ? 0 : p->nghost[2];
    double h = 0.5 * p->dt, Lx = p->L[0], s = shear_offset(p, t), vs = shear_speed(p);
    double margin = 1e-9 * Lx;
    int64_t nitem = n * (int64_t)(ngx + 1);
    orc_stop* st = (orc_stop*)malloc((size_t)(2 * nitem > 0 ? 2 * nitem : 1) * sizeof(orc_stop));
    for (int64_t q = 0; q < nitem; q++) {
        int64_t i = q % n;
        int copy = (int)(q / n);
        double ext = fabs(vx[i]) * h + r[i];
        double xc = x[i] + (double)copy * Lx;
        st[2 * q] = (orc_stop){xc - ext - margin, q, 0};
        st[2 * q + 1] = (orc_stop){xc + ext + margin, q, 1};
    }
    qsort(st, (size_t)(2 * nitem), sizeof(orc_stop), orc_cmp_stop);
    int64_t* list = (int64_t*)malloc((size_t)(nitem > 0 ? nitem : 1) * sizeof(int64_t));
    int64_t* where = (int64_t*)malloc((size_t)(nitem > 0 ? nitem : 1) * sizeof(int64_t));
    int64_t nl = 0, k = 0;
    for (int64_t e = 0; e < 2 * nitem; e++) {
        int64_t q = st[e].item;
        if (st[e].end) { /* remove q from the list (swap with the last) */
            int64_t w = where[q];
            list[w] = list[nl - 1];
            where[list[w]] = w;
            nl--;
            continue;
        }
        for (int64_t l = 0; l < nl; l++) {
            int64_t u = list[l];
            int64_t i = q % n, j = u % n;
            int ci = (int)(q / n), cj = (int)(u / n);
            if ((ci != 0 && cj != 0) || i == j) continue;
            /* image of j as seen from i, then the canonical orientation */
            int gx = cj - ci;
            int64_t a = i, b = j;
            if (id[j] < id[i]) {
                a = j;
                b = i;
                gx = -gx;
            }
            for (int gy = -ngy; gy <= ngy; gy++)
                for (int gz = -ngz; gz <= ngz; gz++) {
                    double o[3] = {(double)gx * Lx, (double)gy * p->L[1] - (double)gx * s,
                                   (double)gz * p->L[2]};
                    if (orc_line_hit(p, a, b, x, y, z, vx, vy, vz, r, o, -(double)gx * vs)) {
                        int code = (gx + 7) | ((gy + 7) << 4) | ((gz + 7) << 8);
                        if (k < cap) keys[k] = orc_pair_key(id[a], id[b], code);
                        k++;
                    }
                }
        }
        list[nl] = q;
        where[q] = nl;
        nl++;
    }
    free(list);
    free(where);
    free(st);
    qsort(keys, (size_t)(k < cap ? k : cap), sizeof(uint64_t), orc_cmp_u64);
    return k;
}

/* Resolution of the collision queue (Sect. 5, Eq. 2; reading R8): pairs in
 * ascending key order; a pair is skipped unless the particles approach; the
 * relative normal velocity is multiplied by -eps and momentum is conserved.
 * Later pairs see the velocities left by earlier ones.  The steps follow the
 * equation: with r = x_b - x_a (ghost offset included) and u = v_b - v_a
 * (ghost shear velocity included), n = r/|r|, v_n = u.n, the change of the
 * normal velocity is Delta = -(1 + eps) v_n, and the two particles share it
 * in inverse proportion to their masses (M = m_a + m_b):
 * v_a -= (m_b/M) Delta n, v_b += (m_a/M) Delta n. */
void orc_resolve(const orc_params* p, double t, int64_t n, const double* x, const double* y,
                 const double* z, double* vx, double* vy, double* vz, const double* m,
                 const int64_t* id, int64_t npairs, const uint64_t* keys) {
    double s = shear_offset(p, t), vs = shear_speed(p);
    int64_t maxid = -1;
    for (int64_t i = 0; i < n; i++) maxid = id[i] > maxid ? id[i] : maxid;
    int64_t* slot = (int64_t*)malloc((size_t)(maxid + 2) * sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) slot[id[i]] = i;
    for (int64_t k = 0; k < npairs; k++) {
        int64_t ia = (int64_t)(keys[k] >> 36), ib = (int64_t)((keys[k] >> 12) & 0xFFFFFF);
        int code = (int)(keys[k] & 0xFFF);
        int gx = (code & 15) - 7, gy = ((code >> 4) & 15) - 7, gz = ((code >> 8) & 15) - 7;
        double o[3] = {(double)gx * p->L[0], (double)gy * p->L[1] - (double)gx * s,
                       (double)gz * p->L[2]};
        double dvg = -(double)gx * vs;
        int64_t a = slot[ia], b = slot[ib];
        double rx = (x[b] + o[0]) - x[a], ry = (y[b] + o[1]) - y[a], rz = (z[b] + o[2]) - z[a];
        double ux = vx[b] - vx[a], uy = (vy[b] + dvg) - vy[a], uz = vz[b] - vz[a];
        double rv = (rx * ux + ry * uy) + rz * uz;
        if (rv >= 0.0) continue; /* not approaching (Sect. 5.1) */
        double rr = sqrt((rx * rx + ry * ry) + rz * rz);
        double nx = rx / rr, ny = ry / rr, nz = rz / rr;
        double vn = (ux * nx + uy * ny) + uz * nz;
        double e = p->eps;
        if (p->eps_law == 1) { /* reading V1 */
            double q = pow(fabs(vn) / p->eps_vc, -p->eps_p);
            e = q < 1.0 ? q : 1.0;
        }
        double dlt = -(1.0 + e) * vn;
        double mt = m[a] + m[b];
        double fa = (m[b] / mt) * dlt, fb = (m[a] / mt) * dlt;
        vx[a] = vx[a] - fa * nx; vy[a] = vy[a] - fa * ny; vz[a] = vz[a] - fa * nz;
        vx[b] = vx[b] + fb * nx; vy[b] = vy[b] + fb * ny; vz[b] = vz[b] + fb * nz;
    }
    free(slot);
}

/* ------------------------------------------------------------------------ */
/* One DKD step (Sect. 3) with gravity (Sect. 4) and collisions (Sect. 5)    */
/* ------------------------------------------------------------------------ */

/* Source masses of Eq. 1 (reading T1): test particles exert no gravity. */
static double* orc_source_mass(const orc_params* p, int64_t n, const double* m, const int64_t* id) {
    double* ms = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    for (int64_t i = 0; i < n; i++)
        ms[i] = (p->n_active >= 0 && id && id[i] >= p->n_active) ? 0.0 : m[i];
    return ms;
}

static void orc_gravity_all(const orc_params* p, double t, int64_t n, const double* x,
                            const double* y, const double* z, const double* m0, const int64_t* id,
                            double* ax, double* ay, double* az, double* phi) {
    double* m = orc_source_mass(p, n, m0, id);
    if (p->gravity == ORC_GRAV_DIRECT) {
        orc_direct_gravity(p, t, n, x, y, z, m, 0, NULL, ax, ay, az, phi);
    } else if (p->gravity == ORC_GRAV_TREE) {
        orc_tree* tr = orc_tree_build(n, x, y, z, m, p->L[0]);
        orc_tree_gravity(tr, p, t, 0, NULL, ax, ay, az, phi, NULL, NULL, NULL);
        orc_tree_free(tr);
    } else {
        for (int64_t i = 0; i < n; i++) {
            ax[i] = ay[i] = az[i] = 0.0;
            if (phi) phi[i] = 0.0;
        }
    }
    free(m);
}

/* Step number `step` (0 = first step after t0): drift dt/2, boundaries,
 * gravity at the mid-step positions, kick dt, drift dt/2, boundaries, then
 * collision detection at the end of the step and resolution (Sect. 5.1:
 * the end of the DKD step is where positions and velocities are in sync).
 * Arrays stay in ascending id order; *n shrinks when particles leave an open
 * box.  Accelerations (when given) are those of the kick, in the array order
 * at kick time; pairs (when given) are the sorted keys found this step. */
int orc_step(const orc_params* p, int64_t step, int64_t* n, double* x, double* y, double* z,
             double* vx, double* vy, double* vz, double* m, double* r, int64_t* id, double* ax,
             double* ay, double* az, int64_t pair_cap, uint64_t* pairs, int64_t* npairs) {
    int64_t N = *n;
    double t1 = orc_time(p, 2 * step + 1), t2 = orc_time(p, 2 * step + 2);
    orc_drift(p, N, x, y, z, vx, vy, vz);
    N = orc_boundary(p, t1, N, x, y, z, vx, vy, vz, m, r, id);
    double* bx = (double*)malloc((size_t)(N > 0 ? N : 1) * 3 * sizeof(double));
    double *gx = bx, *gy = bx + (N > 0 ? N : 1), *gz = bx + 2 * (N > 0 ? N : 1);
    orc_gravity_all(p, t1, N, x, y, z, m, id, gx, gy, gz, NULL);
    orc_kick(p, N, vx, vy, vz, gx, gy, gz);
    if (ax) {
        memcpy(ax, gx, (size_t)N * sizeof(double));
        memcpy(ay, gy, (size_t)N * sizeof(double));
        memcpy(az, gz, (size_t)N * sizeof(double));
    }
    free(bx);
    orc_drift(p, N, x, y, z, vx, vy, vz);
    N = orc_boundary(p, t2, N, x, y, z, vx, vy, vz, m, r, id);
    *n = N;
    int64_t np = 0;
    if (p->collisions != ORC_COLL_NONE) {
        int64_t cap = pair_cap > 0 && pairs ? pair_cap : 4 * N + 16;
        uint64_t* keys = pairs && pair_cap > 0 ? pairs : (uint64_t*)malloc((size_t)cap * sizeof(uint64_t));
        if (p->collisions == ORC_COLL_BRUTE)
            np = orc_collide_brute(p, t2, N, x, y, z, r, id, cap, keys);
        else if (p->collisions == ORC_COLL_SWEEP)
            np = orc_collide_sweep(p, t2, N, x, y, z, vx, vy, vz, r, id, cap, keys);
        else
            np = orc_collide_tree(p, t2, N, x, y, z, r, id, cap, keys);
        if (np > cap) {
            if (keys != pairs) free(keys);
            if (npairs) *npairs = np;
            return -1; /* the pair buffer was too small; state is pre-resolution */
        }
        orc_resolve(p, t2, N, x, y, z, vx, vy, vz, m, id, np, keys);
        if (keys != pairs) free(keys);
    }
    if (npairs) *npairs = np;
    return 0;
}

/* Energy and momentum terms (Sect. 6.2): K = sum m |v|^2 / 2, the Hill
 * tidal and vertical term U = sum m (Omega_z^2 z^2 / 2 - 3/2 Omega^2 x^2)
 * for SEI (0 for leap-frog), W = (1/2) sum m_i phi_i with phi from the same
 * gravity module as the step (tree potential at theta, or direct sum), and
 * P = sum m v.  terms[0..5] = K, U, W, P_x, P_y, P_z. */
void orc_energy_terms(const orc_params* p, double t, int64_t n, const double* x, const double* y,
                      const double* z, const double* vx, const double* vy, const double* vz,
                      const double* m, double* terms) {
    double K = 0.0, U = 0.0, W = 0.0, px = 0.0, py = 0.0, pz = 0.0;
    double O = p->omega, Oz = p->omega_z > 0.0 ? p->omega_z : p->omega;
    for (int64_t i = 0; i < n; i++) {
        double v2 = (vx[i] * vx[i] + vy[i] * vy[i]) + vz[i] * vz[i];
        K = K + 0.5 * m[i] * v2;
        if (p->integrator == ORC_INT_SEI)
            U = U + m[i] * (0.5 * (Oz * Oz) * (z[i] * z[i]) - 1.5 * (O * O) * (x[i] * x[i]));
        px = px + m[i] * vx[i];
        py = py + m[i] * vy[i];
        pz = pz + m[i] * vz[i];
    }
    if (p->gravity != ORC_GRAV_NONE && n > 0) {
        double* buf = (double*)malloc((size_t)n * 4 * sizeof(double));
        orc_gravity_all(p, t, n, x, y, z, m, NULL, buf, buf + n, buf + 2 * n, buf + 3 * n);
        for (int64_t i = 0; i < n; i++) W = W + 0.5 * m[i] * buf[3 * n + i];
        free(buf);
    }
    terms[0] = K; terms[1] = U; terms[2] = W;
    terms[3] = px; terms[4] = py; terms[5] = pz;
}

/* Energy and momentum (Sect. 6.2): E = K + U + W, P = sum m v. */
void orc_energy(const orc_params* p, double t, int64_t n, const double* x, const double* y,
                const double* z, const double* vx, const double* vy, const double* vz,
                const double* m, double* E, double* P) {
    double tm[6];
    orc_energy_terms(p, t, n, x, y, z, vx, vy, vz, m, tm);
    *E = tm[0] + tm[1] + tm[2];
    P[0] = tm[3]; P[1] = tm[4]; P[2] = tm[5];
}
