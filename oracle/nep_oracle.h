/*
 * nep_oracle.h -- interface of the FP64 CPU oracle (test infrastructure only;
 * see nep_oracle.c).  Positions, forces and r_ij are AoS (n x 3), per-atom
 * virials n x 9 row-major (W[9i + 3a + b]), boxes 9 doubles (rows = lattice
 * vectors a, b, c).
 */
#ifndef NEP_ORACLE_H
#define NEP_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_BOX = -2, ORC_ERR_CAPACITY = -3 };

typedef struct {
    int n_max_R; /* radial Chebyshev orders 0..n_max_R, cutoff rc_R */
    int n_max_A; /* angular radial orders 0..n_max_A, cutoff rc_A */
    int l_max;   /* Legendre orders 1..l_max */
    int n_neu;   /* hidden neurons */
    double rc_R;
    double rc_A;
} orc_hyper;

int orc_n_des(const orc_hyper* h);
int orc_n_par(const orc_hyper* h);

void orc_chebyshev(double x, int n, double* T, double* U);
double orc_cutoff(double r, double rc, double* dfc);
void orc_radial(double r, double rc, int nmax, double* g, double* dg);
double orc_legendre(int l, double t, double* dP);

int orc_neighbors(int n, const double* box, const double* pos, double rc, int method, int cap, int* count,
                  int* nbr_j, double* nbr_r);
int orc_descriptors(const orc_hyper* h, int n, const double* box, const double* pos, double* q);
int orc_efv(const orc_hyper* h, const double* z, int n, const double* box, const double* pos, double* U, double* F,
            double* W);
int orc_efv_brute(const orc_hyper* h, const double* z, int n, const double* box, const double* pos, double* U,
                  double* F, double* W);
int orc_efv_sample(const orc_hyper* h, const double* z, int n, const double* box, const double* pos, int n_sample,
                   const int* idx, double* U, double* F, double* W);
int orc_site(const orc_hyper* h, const double* z, int n, const double* box, const double* pos, double* q,
             double* G, double* x);
void orc_heat_current(int n, const double* W, const double* v, double* J);
int orc_md(const orc_hyper* h, const double* z, int n, const double* box, double* pos, double* vel, double mass,
           double dt, int n_steps, double* thermo, double* J);
int orc_md_ext(const orc_hyper* h, const double* z, int n, const double* box, double* pos, double* vel,
               double mass, double dt, int n_steps, double t0, double tau, const double* fe, double* thermo,
               double* J);
int orc_md_record(const orc_hyper* h, const double* z, int n, const double* box, double* pos, double* vel,
                  double mass, double dt, int n_steps, double t0, double tau, const double* fe, const double* Zat,
                  double* thermo, double* J, double* W_hist, double* v_hist);
/* multicomponent weighting: Zat = atomic number of every atom (NULL: one species) */
int orc_descriptors_z(const orc_hyper* h, int n, const double* box, const double* pos, const double* Zat, double* q);
int orc_efv_z(const orc_hyper* h, const double* z, int n, const double* box, const double* pos, const double* Zat,
              double* U, double* F, double* W);
int orc_loss_z(const orc_hyper* h, const double* z, int n_struct, const int* n_atoms, const double* boxes,
               const double* pos, const double* Zat, const double* e_tar, const double* f_tar,
               const double* w_tar, const double* lambdas, double* out);
int orc_force_loss_grad_z(const orc_hyper* h, const double* z, int n_struct, const int* n_atoms,
                          const double* boxes, const double* pos, const double* Zat, const double* f_tar,
                          double* grad, double* lf);
void orc_shc(int n, int n_samples, int n_lags, const double* W_hist, const double* v_hist, double* K_sum);
void orc_shc_spectrum(int n_lags, const double* K, double dt_s, int n_omega, const double* omega, double scale,
                      int window, double* out);
/* kappa(w) x^2 e^x / (e^x - 1)^2 with x = x_per_omega * omega, in place on spec [n_omega][3]. */
void orc_shc_quantum(int n_omega, const double* omega, double x_per_omega, double* spec);
/* Running HNEMD estimate: out[t] = scale * mean of J[0..t] (J, out [n][3]). */
void orc_hnemd_kappa(int n, const double* J, double scale, double* out);
int orc_loss(const orc_hyper* h, const double* z, int n_struct, const int* n_atoms, const double* boxes,
             const double* pos, const double* e_tar, const double* f_tar, const double* w_tar,
             const double* lambdas, double* out);
int orc_force_loss_grad(const orc_hyper* h, const double* z, int n_struct, const int* n_atoms,
                        const double* boxes, const double* pos, const double* f_tar, double* grad, double* lf);
void orc_snes_utilities(int npop, double* u);
double orc_snes_eta_s(int npar);
int orc_snes_update(int npar, int npop, const double* loss, const double* r, double* m, double* s, double eta_m,
                    double eta_s, int* order_out);
void orc_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out);
void orc_gaussian(uint64_t seed, uint32_t gen, long count, double* out);
int orc_num_threads(void);
void orc_set_num_threads(int t);

#ifdef __cplusplus
}
#endif
#endif
