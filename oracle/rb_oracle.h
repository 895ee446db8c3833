/*
 * rb_oracle.h -- interface of the plain FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline leg load this library; the CUDA product path never does, and
 * the two share no code.  Everything is FP64 and is compiled with
 * -ffp-contract=off so each expression is evaluated exactly as written.
 *
 * Conventions (the same conventions are restated, in its own code, by the
 * CUDA path; they are formats both sides must agree on, not shared code):
 *  - root cube: side L = L[0], lower corner -L/2 on every axis (Sect. 2.3);
 *  - integer coordinate per axis: k = floor(((x - lo) / L) * 2^21), clamped
 *    to [0, 2^21 - 1]; the octant at depth d uses bit (20 - d) of k, with the
 *    x bit as the most significant of the three;
 *  - ghost image code: (gx + 7) | (gy + 7) << 4 | (gz + 7) << 8;
 *  - collision pair key: (id_a << 36) | (id_b << 12) | code, id_a < id_b,
 *    code = image of b as seen from a; pairs are resolved in key order.
 */
#ifndef RB_ORACLE_H
#define RB_ORACLE_H
#include <stdint.h>

#define ORC_MAXDEPTH 21

enum { ORC_BC_OPEN = 0, ORC_BC_PERIODIC = 1, ORC_BC_SHEAR = 2 };
enum { ORC_INT_LEAPFROG = 0, ORC_INT_SEI = 1 };
enum { ORC_GRAV_NONE = 0, ORC_GRAV_TREE = 1, ORC_GRAV_DIRECT = 2 };
enum { ORC_COLL_NONE = 0, ORC_COLL_TREE = 1, ORC_COLL_BRUTE = 2, ORC_COLL_SWEEP = 3 };

typedef struct {
    double G, omega, omega_z;   /* omega_z <= 0 means omega_z = omega */
    double L[3];                /* box side per axis */
    double theta, eps, soft, dt, t0;
    int nghost[3];
    int boundary, z_periodic, integrator, quadrupole, gravity, collisions;
    /* test particles (reading T1): ids >= n_active feel gravity but exert
     * none; n_active < 0: every particle is active */
    int64_t n_active;
    /* coefficient of restitution (reading V1): law 0 the constant eps; law 1
     * eps(v_n) = min(1, (|v_n| / eps_vc)^(-eps_p)) */
    int eps_law;
    double eps_vc, eps_p;
} orc_params;

typedef struct orc_tree orc_tree;

const char* orc_version(void);
int  orc_nthreads(void);

/* ghost images at time t; returns the number of images (<= cap) */
int  orc_images(const orc_params* p, double t, int cap, double* off, double* dvy, int* code);
double orc_time(const orc_params* p, int64_t half_step);

/* gravity */
void orc_direct_gravity(const orc_params* p, double t, int64_t n, const double* x, const double* y,
                        const double* z, const double* m, int64_t nt, const int64_t* tsel,
                        double* ax, double* ay, double* az, double* phi);
orc_tree* orc_tree_build(int64_t n, const double* x, const double* y, const double* z,
                         const double* m, double L);
void orc_tree_free(orc_tree* t);
int64_t orc_tree_ncells(const orc_tree* t);
int64_t orc_tree_cells(const orc_tree* t, int64_t cap, int* depth, int64_t* count, int64_t* members,
                       int64_t members_cap, double* M, double* com, double* Q);
void orc_tree_gravity(const orc_tree* t, const orc_params* p, double t_now, int64_t nt,
                      const int64_t* tsel, double* ax, double* ay, double* az, double* phi,
                      int64_t* ncell, int64_t* nleaf, int64_t* nmac);

/* collisions */
int64_t orc_collide_brute(const orc_params* p, double t, int64_t n, const double* x, const double* y,
                          const double* z, const double* r, const int64_t* id, int64_t cap,
                          uint64_t* keys);
int64_t orc_collide_tree(const orc_params* p, double t, int64_t n, const double* x, const double* y,
                         const double* z, const double* r, const int64_t* id, int64_t cap,
                         uint64_t* keys);
int64_t orc_collide_tree_sel(const orc_params* p, double t, int64_t n, const double* x,
                             const double* y, const double* z, const double* r, const int64_t* id,
                             int64_t nt, const int64_t* tsel, int64_t cap, uint64_t* keys);
int64_t orc_tree_collide_sel(const orc_tree* tr, const orc_params* p, double t, int64_t n,
                             const double* x, const double* y, const double* z, const double* r,
                             const int64_t* id, int64_t nt, const int64_t* tsel, int64_t cap,
                             uint64_t* keys);
/* plane sweep (Sect. 5.3): straight-line criterion over tau in [-dt/2, dt/2] */
int64_t orc_collide_line_brute(const orc_params* p, double t, int64_t n, const double* x,
                               const double* y, const double* z, const double* vx, const double* vy,
                               const double* vz, const double* r, const int64_t* id, int64_t cap,
                               uint64_t* keys);
int64_t orc_collide_sweep(const orc_params* p, double t, int64_t n, const double* x,
                          const double* y, const double* z, const double* vx, const double* vy,
                          const double* vz, const double* r, const int64_t* id, int64_t cap,
                          uint64_t* keys);
void orc_resolve(const orc_params* p, double t, int64_t n, const double* x, const double* y,
                 const double* z, double* vx, double* vy, double* vz, const double* m,
                 const int64_t* id, int64_t npairs, const uint64_t* keys);

/* integrators and boundaries */
void orc_drift(const orc_params* p, int64_t n, double* x, double* y, double* z, double* vx,
               double* vy, double* vz);
void orc_kick(const orc_params* p, int64_t n, double* vx, double* vy, double* vz,
              const double* ax, const double* ay, const double* az);
int64_t orc_boundary(const orc_params* p, double t, int64_t n, double* x, double* y, double* z,
                     double* vx, double* vy, double* vz, double* m, double* r, int64_t* id);
int  orc_step(const orc_params* p, int64_t step, int64_t* n, double* x, double* y, double* z,
              double* vx, double* vy, double* vz, double* m, double* r, int64_t* id,
              double* ax, double* ay, double* az, int64_t pair_cap, uint64_t* pairs,
              int64_t* npairs);
void orc_energy(const orc_params* p, double t, int64_t n, const double* x, const double* y,
                const double* z, const double* vx, const double* vy, const double* vz,
                const double* m, double* E, double* P);
/* terms = K, U (SEI tidal + vertical), W, P_x, P_y, P_z */
void orc_energy_terms(const orc_params* p, double t, int64_t n, const double* x, const double* y,
                      const double* z, const double* vx, const double* vy, const double* vz,
                      const double* m, double* terms);

#endif
