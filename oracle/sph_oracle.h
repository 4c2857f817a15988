/*
 * Plain FP64 CPU oracle for the multi-resolution SPH FSI method
 * (arXiv 1911.13255).  TEST INFRASTRUCTURE ONLY: used by the tests, the smoke
 * check and the benchmark's CPU-baseline leg; never by the product path.
 * Arrays are owned by the caller, row-major, in original particle order:
 * vectors n*dim, tensors n*dim*dim.
 */
#ifndef SPH_ORACLE_H
#define SPH_ORACLE_H
#include <stdint.h>

typedef struct {
    int32_t dim;
    int32_t periodic_x;
    double g[3];
    double x_lo, Lx;
    int32_t free_surface;
    int32_t n_reinit;
    int32_t inflow_on;
    int32_t inflow_profile;
    double inflow_width, inflow_y0, inflow_H, inflow_U, inflow_tramp;
    double inflow_period, inflow_wo; /* profile 2: Womersley period T and number Wo */
    double inflow_z0, inflow_Hz;     /* profile 3: the duct's z range [z0, z0 + Hz] */
} or_params;

typedef struct {
    int64_t n;
    double dp, rho0, c0, eta;
    double *r, *v, *rho, *drho, *dvdt;
} or_fluid;

typedef struct {
    int64_t n;
    double dp;
    double *r, *nrm;
} or_wall;

typedef struct {
    int64_t n;
    double dp, rho0, E, nu;
    const uint8_t *cons;
    double *r0, *n0, *r, *v, *F, *Fdot, *B0, *nrm, *vbar, *abar, *fF;
    int64_t *nb_ptr, *nb_idx;
} or_solid;

typedef struct {
    int64_t n_ff, n_fw, n_fs, n_sf, n_ss;
    double vmax_f, vmax_s, amax_s;
    double mom_fs_fluid[3], mom_fs_solid[3], abs_fs;
} or_diag;

int or_threads(void);
double or_kernel_W(int dim, double r, double h);
double or_kernel_dW(int dim, double r, double h);
double or_lattice_sigma0(int dim, double dp, double h);
double or_eos_p(double rho, double rho0, double c0);
double or_eos_rho(double p, double rho0, double c0);
double or_riemann(int dim, const double *e, const double *vL, const double *vR, double pL, double pR,
                  double rhoL, double rhoR, double c0, double *vstar);
void or_neo_hookean_P(int dim, const double *F, double mu, double lam, double *Pout);
double or_solid_sound_speed(double E, double nu, double rho0);
int64_t or_pairs_count(const or_params *P, int dim, const double *A, int64_t nA, const double *B, int64_t nB,
                       double rc, int same, int brute);
int or_pairs_fill(const or_params *P, int dim, const double *A, int64_t nA, const double *B, int64_t nB,
                  double rc, int same, int brute, int64_t *ptr, int64_t *idx);
int64_t or_solid_count(const or_params *P, const or_solid *s);
int or_solid_setup(const or_params *P, or_solid *s);
int or_solid_F_from_positions(const or_params *P, const or_solid *s, double *Fout);
int or_solid_accel(const or_params *P, const or_solid *s, const double *F, double *acc);
double or_inflow_u(const or_params *P, double y, double t);
double or_inflow_u3(const or_params *P, double y, double z, double t);
int or_step(const or_params *P, or_fluid *f, const or_wall *w, or_solid *s, double dt, int K, double t,
            int64_t step_index, or_diag *dg);
/* Pair configuration frozen over the acoustic steps of one advection step
 * (Algorithm 1, reading F2): the neighbour lists and the fluid and solid
 * positions that every pair's kernel value and gradient are evaluated at.
 * valid = 0 makes the next or_step_ex build it at its mid state. */
typedef struct {
    int32_t valid;
    int64_t nf, ns;
    void *lists;
    double *fr, *sr;
} or_cache;
int or_step_ex(const or_params *P, or_fluid *f, const or_wall *w, or_solid *s, double dt, int K, double t,
               int64_t step_index, or_diag *dg, or_cache *c);
void or_cache_free(or_cache *c);
void or_suggest_dt(const or_params *P, const or_fluid *f, const or_solid *s, double vmax_f, double vmax_s,
                   double amax_s, double *dt_ac, double *dt_ad, double *dt_s);
int or_substeps(double dt_f, double dt_s);
double or_single_dt(const or_params *P, const or_fluid *f, const or_solid *s, int mode, double vmax_f,
                    double vmax_s, double amax_s);
void or_eos_rho_array(int64_t n, const double *p, double *rho, double rho0, double c0);
#endif
