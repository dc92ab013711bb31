/* pdf_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, single-threaded FP64 CPU oracle of the per-particle time step
 * of the particle-in-cell joint velocity-frequency-scalar PDF method of
 * Bakosi, Franzese & Boybeyi, "Joint PDF modelling of turbulent flow and
 * dispersion in an urban street canyon" (Section 2, Eqs. Lagrangian-position,
 * Lagrangian-velocity, IECM, dissipation, frequency-model, frequency_source,
 * micromixing-timescale, Gij, C0, elliptic-relaxation, H, L, wall-GandC,
 * wall-normal-velocity ... wall-omega; Section 3).
 *
 * Only the test-suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this library. It shares no code, header, helper or constant table
 * with the CUDA library; the product path never calls it.
 */
#ifndef PDF_ORACLE_H
#define PDF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_params {
    /* Table 2 */
    double C1, C2, C3, C4, CT, CL, Ceta, Cv, gamma5, Comega1, Comega2, Cs, Ct;
    /* Section 2.2: SLM constant, log-law constants */
    double C0, Cmu, kappa, E;
    double nu;              /* kinematic viscosity */
    double fx, fy;          /* imposed -(1/rho) d<P>/dx_i */
    double yp;              /* wall-function distance y_p */
    double wall_offset;     /* distance from the mesh wall to the physical wall */
    double x0, y0, r0;      /* scalar source centre and radius */
    double period;          /* periodic length in x */
    double k0, ustar, y_roof; /* initial condition */
    double er_wall;         /* wall value coefficient: wp_ij = -er_wall*eps*n_i*n_j */
    double floor_k, floor_eps, floor_omega;
    double cg_tol;
    int32_t cg_maxit;
    int32_t nb1, nb2, nb3;  /* velocity bins per direction */
    int32_t wall_model;     /* 0 wall functions (SLM), 1 elliptic relaxation */
    int32_t mix_exp;        /* 0 Euler r = dt/tm, 1 r = 1 - exp(-dt/tm) */
    int32_t reflect_max;
    int32_t rotta;          /* 1: drop the H_ijkl term (Section 4 variant) */
    uint64_t seed;
    uint32_t case_id;
    int32_t omega_wall;     /* 1: Section 4 frequency reflection with <omega v>/<omega v^2> */
    int32_t pressure;       /* 1: mean-pressure projection after each step (see orc_project) */
    int32_t pad_;
} orc_params;

typedef struct orc_ctx orc_ctx;

enum {
    ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_MESH = -2, ORC_ERR_LOST = -5,
    ORC_ERR_WALL = -6, ORC_ERR_CG = -7, ORC_ERR_DT = -8, ORC_ERR_STATE = -9
};

/* field ids for orc_get_field (doubles, row-major) */
enum {
    ORC_F_ELEM_N = 0,      /* ntri            particle count */
    ORC_F_ELEM_MEAN = 1,   /* ntri x 5        <U>,<V>,<W>,<psi>,<omega> */
    ORC_F_ELEM_R = 2,      /* ntri x 6        uu,vv,ww,uv,uw,vw (central, 1/n) */
    ORC_F_ELEM_PSIVAR = 3, /* ntri            psi variance */
    ORC_F_ELEM_CM = 4,     /* ntri x B        <phi|V> per bin */
    ORC_F_NODE_MEAN = 5,   /* nnode x 4       <U>,<V>,<psi>,<omega> */
    ORC_F_NODE_R = 6,      /* nnode x 6 */
    ORC_F_NODE_KE = 7,     /* nnode x 2       k, eps (floored) */
    ORC_F_ELEM_DER = 8,    /* ntri x 9        Ux,Uy,Vx,Vy, lapU,lapV, S_omega, t_m, L */
    ORC_F_NODE_PACK = 9,   /* nnode x 11      U,V,Om,C0eps,G11,G12,G21,G22,G33,Fx,Fy */
    ORC_F_NODE_WP = 10,    /* nnode x 5       wp11,wp12,wp21,wp22,wp33 */
    ORC_F_NODE_WDIST = 11, /* nnode           wall distance */
    ORC_F_NODE_GRAD = 12,  /* nnode x 4       recovered grad <U> */
    ORC_F_NODE_PSIVAR = 13, /* nnode */
    ORC_F_ELEM_OMW = 14,   /* ntri x 5        <omega u>,<omega v>,<omega uu>,<omega uv>,<omega vv> */
    ORC_F_NODE_OMW = 15,   /* nnode x 5 */
    ORC_F_NODE_P = 16      /* nnode           projection pressure p (pressure = 1) */
};

orc_ctx* orc_create(const orc_params* p, int32_t nnode, const double* xy, int32_t ntri,
                    const int32_t* tri, const int32_t* edge_tag, const int32_t* periodic_pair,
                    int32_t* status);
void orc_destroy(orc_ctx* c);
int32_t orc_num_particles(const orc_ctx* c);
int32_t orc_step_index(const orc_ctx* c);
int orc_seed(orc_ctx* c, int32_t per_element);
int orc_set_particles(orc_ctx* c, int32_t n, const double* x, const double* y, const double* u,
                      const double* v, const double* w, const double* om, const double* psi,
                      const uint32_t* id, const int32_t* elem, int32_t step);
int orc_get_particles(const orc_ctx* c, double* x, double* y, double* u, double* v, double* w,
                      double* om, double* psi, uint32_t* id, int32_t* elem, uint8_t* bin);
int orc_estimate_stats(orc_ctx* c);
int orc_advance(orc_ctx* c, double dt);   /* particles only, fields from current stats */
int orc_step(orc_ctx* c, double dt, int32_t nsteps); /* advance + re-estimate, nsteps times */
int orc_advance_subset(orc_ctx* c, double dt, const int32_t* idx, int32_t n);
int orc_get_field(const orc_ctx* c, int32_t field, double* out);
int32_t orc_cg_iterations(const orc_ctx* c);

/* Time averages, probes and scalar CDFs (Section 3, Table 1, Fig. 7): while
 * averaging is on, every orc_step adds its element and node statistics to
 * running sums and the psi of the particles in each CDF point's element to
 * that point's histogram (nbins equal bins on [0, 1]). */
int orc_set_averaging(orc_ctx* c, int32_t on, int32_t reset);
int32_t orc_averaging_count(const orc_ctx* c);
int orc_get_averages(const orc_ctx* c, int32_t which, double* out);
int orc_probe(const orc_ctx* c, int32_t which, int32_t comp, const double* x, const double* y, int32_t n,
              double* out, int32_t* elem_out);
int orc_set_cdf_probes(orc_ctx* c, const double* x, const double* y, int32_t n, int32_t nbins);
int orc_get_cdf(const orc_ctx* c, double* out, int32_t* elem_out);

/* test hooks (pins) */
void orc_philox4x32_10(const uint32_t key[2], const uint32_t ctr[4], uint32_t out[4]);
void orc_gauss8(uint64_t seed, uint32_t case_id, uint32_t id, uint32_t step, double z[8]);
int32_t orc_locate(const orc_ctx* c, double x, double y);
int orc_reflect(const orc_ctx* c, int32_t tag, const double n[2], const double stat[12],
                double* u, double* v, double* w, double* om);
/* Mean-pressure projection of the particle velocities over a step dt (the
 * element statistics must be current): solves the P1 Galerkin pressure
 * problem K p = (1/dt) D <U>, corrects U_p -= dt grad p, and re-estimates
 * the statistics. */
int orc_project(orc_ctx* c, double dt);
void orc_sde(const orc_params* p, int32_t n, double dt, const double* fields, const double* z,
             double* u, double* v, double* w, double* om, double* psi);
int orc_fe_solve(orc_ctx* c, const double* L_elem, const double* f_node, const double* g_node,
                 const uint8_t* is_dir, double* x_out, int32_t ncomp);
int orc_bins(const orc_params* p, int32_t n, const double* u, const double* v, const double* w,
             const uint32_t* id, int32_t* bin);
int orc_set_node_fields(orc_ctx* c, const double* nmean, const double* nR, const double* nke);
int orc_set_node_wp(orc_ctx* c, const double* wp);
int orc_h_contract(const orc_params* p, const double R[6], const double g[4], double k,
                   double om, double f[5]);

#ifdef __cplusplus
}
#endif
#endif
