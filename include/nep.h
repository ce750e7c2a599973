/*
 * nep.h -- C ABI of the GB300 (sm_103a) neuroevolution-potential library.
 *
 * The method is the NEP of Fan et al., "Neuroevolution machine learning
 * potentials" (arXiv 2107.08119).  Equation numbers below are the paper's.
 *
 * Conventions for every entry point
 *   - Return value: NEP_OK (0) or a negative nep_status; never aborts or
 *     throws across the ABI.  nep_last_error() gives a message for the last
 *     failing call of the calling thread.
 *   - "dev" pointers are CUDA device memory owned by the caller; "host"
 *     pointers are ordinary host memory read during the call only.
 *   - Work is enqueued on the caller's CUDA stream (cudaStream_t passed as
 *     void*, NULL = legacy default stream) and is asynchronous; errors found
 *     on the device (neighbour-list overflow, non-finite values) are latched
 *     in the handle and reported by nep_sync_status().
 *   - Units: Angstrom, eV, amu, fs.  Positions and velocities are FP64
 *     structure-of-arrays [3][n] (all x, then all y, then all z).  Per-atom
 *     forces and virials are FP32; site energies and totals are FP64.
 *   - Boxes are 9 doubles, rows = lattice vectors a, b, c.  This library
 *     handles orthorhombic boxes (a, b, c along x, y, z); each edge must be
 *     at least half the neighbour-list radius.  Other boxes: NEP_ERR_BOX.
 *   - Handles are not thread-safe: one handle, one host thread at a time.
 */
#ifndef NEP_H
#define NEP_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NEP_OK = 0,
    NEP_ERR_ARG = -1,                /* null pointer, bad size, bad hyperparameter */
    NEP_ERR_OOM = -2,                /* device allocation failed */
    NEP_ERR_CUDA = -3,               /* a CUDA runtime call failed */
    NEP_ERR_NEIGHBOR_OVERFLOW = -4,  /* an atom had more than max_neighbors neighbours */
    NEP_ERR_NONFINITE = -5,          /* non-finite site energy or force */
    NEP_ERR_TIMEOUT = -6,            /* a bounded device-side wait gave up */
    NEP_ERR_BOX = -7,                /* box not orthorhombic, or an edge too short */
    NEP_ERR_UNSUPPORTED = -8         /* hyperparameters this build has no kernel for */
} nep_status;

/*
 * Hyperparameters (Table I of the paper names n_max^R, n_max^A, l_max, N_neu,
 * r_c^R, r_c^A).  Descriptor size N_des = (n_max_R+1) + (n_max_A+1) l_max
 * (Eq. 16); parameter count N_par = (N_des+2) N_neu + 1 (Eq. 26).
 * This build has kernels for n_max_R = 7, n_max_A = 5, l_max = 4 and any
 * n_neu in [1, 64].
 */
typedef struct {
    int n_max_R;        /* radial Chebyshev orders 0..n_max_R */
    int n_max_A;        /* radial orders 0..n_max_A inside the angular terms */
    int l_max;          /* Legendre orders 1..l_max */
    int n_neu;          /* hidden-layer neurons */
    double rc_R;        /* radial cutoff r_c^R */
    double rc_A;        /* angular cutoff r_c^A */
    double skin;        /* Verlet skin for MD; the list radius is max(rc_R, rc_A) + skin */
    int max_neighbors;  /* Verlet-list capacity per atom, 1..384 (e.g. 96) */
} nep_hyper;

typedef struct nep_model nep_model;
typedef struct nep_md nep_md;

/*
 * nep_create -- build a model handle.
 *   hp      host, hyperparameters (copied).
 *   z       host, n_par floats: the parameter vector of Sec. II.D.3,
 *           laid out as w1 [n_neu][N_des] row-major, b1 [n_neu], w2 [n_neu], b2,
 *           with descriptor order q_0..q_{n_max_R}, then q_{nl} with n outer and
 *           l inner.  Biases enter with a minus sign (Eqs. 21-22).
 *   out     receives the handle; the handle owns all device scratch.
 * Errors: NEP_ERR_ARG, NEP_ERR_UNSUPPORTED, NEP_ERR_OOM, NEP_ERR_CUDA.
 */
int nep_create(const nep_hyper* hp, const float* z, int n_par, nep_model** out);

/* Replace the parameter vector (host, n_par floats); stream-ordered copy. */
int nep_set_parameters(nep_model* m, const float* z, int n_par, void* stream);

/* Free the handle and its device scratch (synchronises the device). */
int nep_destroy(nep_model* m);

/*
 * nep_compute_efv -- site energies, forces and per-atom virials of one
 * configuration (Sec. II.A-D):
 *   U_i (Eq. 22) from the descriptor q^i (Eqs. 12-15) through the network
 *   (Eqs. 21-22); partial forces dU_i/dr_ij (Eqs. 23-25); forces
 *   F_i = sum_j (dU_i/dr_ij - dU_j/dr_ji) (Eqs. 4-5); per-atom virials
 *   W_i^{ab} = sum_j r_ij^a (dU_j/dr_ji)^b (Eq. 6).
 *   n            number of atoms, 1 <= n < 2^24.
 *   box9         host, 9 doubles (orthorhombic).
 *   pos          dev, FP64 [3][n]; not modified (wrapped into the box internally).
 *   e_total      dev, 1 double, sum_i U_i; or NULL.
 *   e_atom       dev, n doubles, U_i (the FP32 path carries U_i as a compensated
 *                hi + lo pair; it is reported without a final FP32 rounding); or NULL.
 *   force        dev, FP32 [3][n]; or NULL.
 *   virial_atom  dev, FP32 [9][n], component 3a+b holds W_i^{ab}; or NULL.
 *   virial_total dev, 9 doubles, sum_i W_i (symmetric); or NULL.
 *   stream       cudaStream_t.
 * The neighbour list is rebuilt on every call with radius max(rc_R, rc_A).
 * Errors: NEP_ERR_ARG, NEP_ERR_BOX, NEP_ERR_OOM, NEP_ERR_CUDA (immediate);
 * NEP_ERR_NEIGHBOR_OVERFLOW (latched, see nep_sync_status).
 */
int nep_compute_efv(nep_model* m, int n, const double* box9, const double* pos, double* e_total, double* e_atom,
                    float* force, float* virial_atom, double* virial_total, void* stream);

/*
 * nep_compute_efv_plain -- the same outputs as nep_compute_efv, computed by
 * the plain FP32 GPU form that the optimised path is measured against: one
 * thread per atom, three unfused passes (descriptors, network, partial
 * forces), q_nl by the literal double sum over neighbour pairs of Eq. 13 with
 * Legendre polynomials (O(M^2) per atom), partial forces by Eqs. 24-25, and
 * no compensated sums (so site energies carry plain FP32 rounding, ~1e-5 eV).
 * It shares the neighbour list, assembly and reductions with nep_compute_efv.
 * At most 96 neighbours within r_c^A per atom (NEP_ERR_NEIGHBOR_OVERFLOW,
 * latched).  Same arguments and errors as nep_compute_efv.
 */
int nep_compute_efv_plain(nep_model* m, int n, const double* box9, const double* pos, double* e_total,
                          double* e_atom, float* force, float* virial_atom, double* virial_total, void* stream);

/*
 * nep_sync_status -- synchronise `stream`, then return and clear the first
 * device-side error latched by earlier calls on this handle (NEP_OK if none).
 */
int nep_sync_status(nep_model* m, void* stream);

/*
 * nep_heat_current -- J = sum_i W_i . v_i, J^a = sum_b W_i^{ab} v_i^b
 * (Eq. 7 summed over atoms), products in FP32 and accumulation in FP64, in a
 * fixed order (deterministic).
 *   virial_atom  dev, FP32 [9][n] as written by nep_compute_efv.
 *   vel          dev, FP64 [3][n] (Angstrom/fs).
 *   J            dev, 3 doubles (eV Angstrom/fs).
 */
int nep_heat_current(nep_model* m, int n, const float* virial_atom, const double* vel, double* J, void* stream);

/*
 * Molecular dynamics: NVE velocity Verlet with a Verlet neighbour list of
 * radius max(rc_R, rc_A) + skin, rebuilt on the device whenever an atom has
 * moved more than skin/2 since the last build.  Per step:
 *   v += dt/2 F/m; x += dt v; [rebuild]; F, W from x; v += dt/2 F/m;
 *   then E_pot, E_kin, sum_i W_i and J = sum_i W_i . v_i (Eq. 7) in FP64.
 * Positions, velocities and the integrator update are FP64; the force path
 * is FP32.  Positions are wrapped into the box at every list rebuild.
 *
 * nep_md_create: n atoms of one species of mass `mass` (amu) in box9 (host).
 */
int nep_md_create(nep_model* m, int n, const double* box9, double mass, nep_md** out);
int nep_md_destroy(nep_md* md);

#define NEP_THERMO_COLS 8 /* E_pot, E_kin, W_xx, W_yy, W_zz, W_xy, W_yz, W_zx (eV) */

/*
 * nep_md_step -- advance n_steps steps of dt fs.
 *   pos, vel   dev, FP64 [3][n], updated in place.
 *   thermo     dev, [n_steps][NEP_THERMO_COLS] doubles, or NULL.
 *   heat       dev, [n_steps][3] doubles: J after each step, or NULL.
 * Forces are recomputed at the start of a call when the positions may have
 * changed outside the library (first call, or nep_md_invalidate()).
 */
int nep_md_step(nep_md* md, double* pos, double* vel, int n_steps, double dt, double* thermo, double* heat,
                void* stream);

/* Mark positions as changed by the caller: the next step rebuilds the list and forces. */
int nep_md_invalidate(nep_md* md);

/*
 * nep_md_set_thermostat -- Berendsen velocity rescaling for the following
 * steps: after the second half kick and the heat current of each step,
 * v *= lambda with lambda^2 = 1 + (dt/tau)(T0/T - 1) and T = 2 E_kin /
 * ((3N - 3) k_B); the thermo row then reports E_kin after the rescaling, J
 * before it.  The paper runs its speed benchmark in the NVT ensemble without
 * naming a thermostat (Sec. III.C); this is the simplest deterministic one.
 *   t0   target temperature (K), >= 0.   tau  coupling time (fs); <= 0: off (NVE).
 * Errors: NEP_ERR_ARG.  nep_md_step needs n >= 2 while it is on.
 */
int nep_md_set_thermostat(nep_md* md, double t0, double tau);

/*
 * nep_md_set_force_form -- which form of the force pass the MD steps use:
 * NEP_FORCE_OPTIMISED (the default: the O(M) harmonic form of Eq. 13 with
 * compensated sums, as nep_compute_efv) or NEP_FORCE_PLAIN_FP32 (the plain
 * comparator of nep_compute_efv_plain: literal O(M^2) Eq. 13, unfused, plain
 * FP32 sums; at most 96 neighbours within r_c^A).  Everything else in the
 * step (list, assembly, integrator, heat current) is shared.  The next step
 * recomputes the starting forces with the selected form.  The plain form
 * allocates 256 bytes per atom of scratch on first use.
 * Errors: NEP_ERR_ARG (unknown form), NEP_ERR_OOM.
 */
#define NEP_FORCE_OPTIMISED 0
#define NEP_FORCE_PLAIN_FP32 1
int nep_md_set_force_form(nep_md* md, int form);

/*
 * nep_set_species -- multicomponent systems (Sec. II.A): the cutoff function
 * of pair (i, j) becomes f_c(r_ij) sqrt(Z_i Z_j), so every g_n and g_n' of
 * the pair is multiplied by sqrt(Z_i Z_j) (one species: weight 1, the default).
 *   n       atoms of the configurations that follow (0: back to one species).
 *   z_atom  host [n] species numbers (atomic numbers, > 0).
 * Later nep_compute_efv calls and MD handles created afterwards for n atoms
 * use them (a call for another atom count fails with NEP_ERR_ARG); the plain
 * comparator (nep_compute_efv_plain) and nep_compute_efv_static stay one
 * species.  Synchronises the device.
 * Errors: NEP_ERR_ARG (NULL, non-positive Z), NEP_ERR_OOM, NEP_ERR_CUDA.
 */
int nep_set_species(nep_model* m, int n, const double* z_atom);

/*
 * nep_md_set_hnemd -- homogeneous non-equilibrium MD driving (Sec. II.B):
 * every atom feels F_i^ext = F_e . W_i, (F_i^ext)^b = sum_a F_e^a W_i^{ab},
 * minus its mean over all atoms so that the total momentum is kept; then
 * <J>/(T V) = kappa F_e gives the thermal conductivity.  With the drive on,
 * each step assembles F and W_i, sums W, and applies the second half kick
 * with F + F^ext in a separate kernel; the forces the next step starts from
 * (and nep_md_forces) include F^ext.
 *   fe   host [3] driving force parameter (1/A), or NULL / all zero: off.
 * The next nep_md_step recomputes the starting forces.
 * Errors: NEP_ERR_ARG, NEP_ERR_OOM.
 */
int nep_md_set_hnemd(nep_md* md, const double* fe);

/*
 * nep_md_set_shc -- spectral heat current (Sec. II.B): accumulate the
 * virial-velocity correlation K(t) = sum_i < W_i(0) . v_i(t) >, with
 * (W . v)^a = sum_b W^{ab} v^b as in Eq. 7, during nep_md_step.  Every
 * `every`-th step (counted from this call, across nep_md_step calls) is a
 * sample s: W_i of that step goes into a ring of n_lags samples and, with
 * v_i(s) taken where J is (after the second half kick, before a thermostat),
 * sum_i W_i(s - tau) . v_i(s) is added to K[tau] for 0 <= tau < min(s + 1,
 * n_lags), in FP64 and a fixed order.  Memory: 36 n n_lags bytes of ring.
 *   n_lags  0 (off: frees the buffers) or 1..100000; every >= 1.
 * Resets the sums.  Errors: NEP_ERR_ARG, NEP_ERR_OOM.
 */
int nep_md_set_shc(nep_md* md, int n_lags, int every);
/*
 * nep_md_get_shc -- K[tau] (dev [n_lags][3] FP64, or NULL) = the sum for lag
 * tau over the samples so far divided by its number of time origins
 * (n_samples - tau; 0 where there is none), and the number of samples
 * (host, or NULL).  Stream-ordered after the steps on `stream`.
 * Errors: NEP_ERR_ARG (NULL handle, correlation off), NEP_ERR_CUDA.
 */
int nep_md_get_shc(nep_md* md, double* K, long long* n_samples, void* stream);
/*
 * nep_shc_spectrum -- the transform of Sec. II.B, (2/(T V)) int K(t) e^{iwt} dt
 * = sum_nu kappa_{mu nu}(w) F_e^nu, for K known at t = tau dt_lag,
 * 0 <= tau < n_lags, and even in t: out[k][a] = scale * 2 * (trapezoid of
 * K[tau][a] cos(omega_k tau dt_lag) over the lags), with K first multiplied by
 * the Hann window (1 + cos(pi tau / (n_lags - 1))) / 2 when window != 0.
 * scale = 2 / (T V F_e) gives kappa(w) in the units of K dt / (T V F_e).
 *   K dev [n_lags][3]; omega dev [n_omega] (rad per unit of dt_lag);
 *   out dev [n_omega][3].  All FP64.
 * Errors: NEP_ERR_ARG, NEP_ERR_CUDA.
 */
int nep_shc_spectrum(const double* K, int n_lags, double dt_lag, int n_omega, const double* omega, double scale,
                     int window, double* out, void* stream);
/*
 * nep_shc_quantum -- the quantum correction of a classical spectral
 * conductivity (Sec. IV.C): spec[k][a] *= x^2 e^x / (e^x - 1)^2 with
 * x = x_per_omega * omega[k] (x_per_omega = hbar / (k_B T) in the time unit of
 * 1/omega), in place; 1 at omega = 0, even in omega.
 *   omega dev [n_omega]; spec dev [n_omega][3].  All FP64.
 * Errors: NEP_ERR_ARG (NULL pointers, n_omega < 1, x_per_omega not finite),
 * NEP_ERR_CUDA.
 */
int nep_shc_quantum(const double* omega, int n_omega, double x_per_omega, double* spec, void* stream);
/*
 * nep_hnemd_kappa -- running HNEMD conductivity estimate (Sec. II.B):
 * <J>/(T V) = kappa F_e, so out[t][a] = scale * (sum_{s<=t} J[s][a]) / (t+1)
 * with scale = 1 / (T V F_e) in the caller's units.  The sums are FP64 in a
 * fixed order (contiguous segments, then their prefix), so the result is
 * reproducible bit for bit.
 *   J dev [n][3] (e.g. the heat series of nep_md_step); out dev [n][3].
 * Errors: NEP_ERR_ARG (NULL pointers, n < 1), NEP_ERR_CUDA.
 */
int nep_hnemd_kappa(const double* J, int n, double scale, double* out, void* stream);
/*
 * nep_hnemd_kappa_si -- nep_hnemd_kappa in physical units: out[t][a] =
 * <J^a>_{0..t} / (T V F_e) in W / (m K), for J in eV A/fs (the heat series
 * of nep_md_step), temperature T in K, volume V in A^3 and the driving force
 * component fe (1/A) along the direction of interest (Sec. II.B; 1 eV/(A fs K)
 * = 1.602176634e6 W/(m K)).
 * Errors: NEP_ERR_ARG (NULL pointers, n < 1, T or V not positive, fe = 0,
 * non-finite values), NEP_ERR_CUDA.
 */
int nep_hnemd_kappa_si(const double* J, int n, double temperature, double volume, double fe, double* out,
                       void* stream);
/*
 * nep_kappa_spectrum -- the spectral conductivity of Sec. II.B in physical
 * units: kappa(nu) in W / (m K THz) at the frequencies nu (THz) from the
 * virial-velocity correlation K (eV A/fs, as nep_md_get_shc returns it) at
 * lags dt_lag_fs apart: omega = 2 pi nu (rad/fs) and
 * kappa(omega) = (2 / (T V F_e)) int K(t) cos(omega t) dt as nep_shc_spectrum
 * computes it (trapezoid over the lags, optional Hann window), expressed per
 * THz of nu so that int kappa(nu) dnu is the HNEMD conductivity.  quantum != 0
 * applies the correction of Sec. IV.C at temperature T (nep_shc_quantum with
 * x = hbar omega / k_B T, hbar = 0.6582119569 eV fs).
 *   K dev [n_lags][3]; nu_thz dev [n_nu]; out dev [n_nu][3].  All FP64.
 * Errors: NEP_ERR_ARG (NULL pointers, empty lengths, dt, T or V not positive,
 * fe = 0), NEP_ERR_CUDA.
 */
int nep_kappa_spectrum(const double* K, int n_lags, double dt_lag_fs, const double* nu_thz, int n_nu,
                       double temperature, double volume, double fe, int window, int quantum, double* out,
                       void* stream);

/* Number of neighbour-list builds so far (synchronises `stream`). */
int nep_md_rebuild_count(nep_md* md, long long* count, void* stream);

/* Per-atom force (FP32 [3][n], dev) of the current MD state, owned by the handle. */
const float* nep_md_forces(const nep_md* md);

/*
 * nep_get_neighbors -- copy the neighbour list built by the last
 * nep_compute_efv call on this handle (radius max(rc_R, rc_A)).
 *   count  dev, n ints: neighbours of each atom (may exceed max_neighbors
 *          when the list overflowed).
 *   nbr    dev, [max_neighbors][n] ints, slot-major: entry (k, i) is
 *          j | c << 24 for the k-th neighbour j of atom i seen through the
 *          periodic image (sx, sy, sz) = (c/25 - 2, (c/5)%5 - 2, c%5 - 2),
 *          i.e. r_ij = r_j + sx a + sy b + sz c - r_i.  Slots beyond count
 *          are unspecified.  Order: increasing distance (ties keep the cell
 *          stencil / atom index order).
 */
int nep_get_neighbors(nep_model* m, int n, int* count, int* nbr, void* stream);

/*
 * nep_status_from_bits -- the status that device-side error bits stand for
 * (host only; no CUDA call).  The kernels latch these bits in a handle (read
 * by nep_sync_status) or, for nep_compute_efv_static, in its err_out word:
 *   1  an atom had more neighbours than max_neighbors  -> NEP_ERR_NEIGHBOR_OVERFLOW
 *   4  a reverse pair was missing (asymmetric list)    -> NEP_ERR_NEIGHBOR_OVERFLOW
 *   2  a non-finite position, site energy or force     -> NEP_ERR_NONFINITE
 *   8  a bounded device-side wait gave up              -> NEP_ERR_TIMEOUT
 * With several bits set the first in that order wins; 0 gives NEP_OK.  Sets
 * the thread's nep_last_error message.
 */
int nep_status_from_bits(unsigned bits);

/*
 * nep_cell_grid -- the cell grid the neighbour-list build uses for a box and
 * list radius (host only; no CUDA call).  Each direction gets floor(L / r_list)
 * cells, so every cell edge is at least r_list and the 27 cells around an
 * atom's cell hold all its neighbours.  A grid of more than 2^22 cells (a
 * large, sparse box) is coarsened by halving its longest direction until it
 * fits; edges only grow, so the list stays exact.  Boxes with fewer than 3
 * cells in some direction use the all-pairs search, reported as 0 0 0.
 *   box9    host, 9 doubles (orthorhombic).
 *   r_list  list radius (Angstrom), > 0.
 *   nc      host, 3 ints: cells per direction.
 * Errors: NEP_ERR_ARG, NEP_ERR_BOX (as nep_compute_efv).
 */
int nep_cell_grid(const double* box9, double r_list, int* nc);

/*
 * Training set for the separable natural evolution strategy (Sec. II.D.2):
 * structures of uneven size evaluated together (Sec. II.E concatenates them
 * into one "super-structure").  nep_dataset_create copies the structures to
 * the device and precomputes everything independent of the parameters:
 * descriptors and, per pair, the derivatives of each atom's descriptor with
 * respect to its pair vectors (Eqs. 24-25).
 *   n_struct   number of structures (>= 1); n_atoms host [n_struct].
 *   boxes      host [n_struct][9] (orthorhombic).
 *   pos        host [N][3] FP64 (AoS; structures consecutive), N = sum n_atoms.
 *   e_tar      host [n_struct] target energies (eV, per structure).
 *   f_tar      host [N][3] target forces (eV/A).
 *   w_tar      host [n_struct][6] target virials sum_i W_i, order xx yy zz xy yz zx.
 * The handle keeps a pointer to the model (same hyperparameters).
 */
typedef struct nep_dataset nep_dataset;
int nep_dataset_create(nep_model* m, int n_struct, const int* n_atoms, const double* boxes, const double* pos,
                       const double* e_tar, const double* f_tar, const double* w_tar, nep_dataset** out);
/* nep_dataset_create for a multicomponent set: z_atom host [N] species
 * numbers (atomic numbers, > 0; NULL = one species), see nep_set_species. */
int nep_dataset_create_species(nep_model* m, int n_struct, const int* n_atoms, const double* boxes,
                               const double* pos, const double* z_atom, const double* e_tar, const double* f_tar,
                               const double* w_tar, nep_dataset** out);
int nep_dataset_destroy(nep_dataset* ds);
/* Atoms, stored pairs and device bytes of a training set; pointers may be NULL. */
int nep_dataset_info(const nep_dataset* ds, int* n_atoms, long long* n_pairs, long long* device_bytes);
/* Sizes of a training set, host long long[5]: atoms, stored pairs (within
 * max(r_c^R, r_c^A)), angular pairs (within r_c^A), structures, atoms of the
 * largest structure. */
int nep_dataset_counts(const nep_dataset* ds, long long* counts);
/* Copy the precomputed descriptors, dev [N][N_des] FP32. */
int nep_dataset_descriptors(const nep_dataset* ds, float* q, void* stream);

/*
 * Launch shape of the population evaluation of a dataset, host int[8]:
 *   [5] fused       0, 4, 8 or 16.  Nonzero: the fused contraction, one
 *                   block per (structure, group of this many members), the
 *                   structure's forces summed in shared memory (exactly, as
 *                   int32 fixed point on 2^-8 and 2^-32 grids) and its loss
 *                   sums written directly: no per-pair partial forces in
 *                   device memory.  Needs (atoms of the largest structure) x
 *                   members x 48 bytes of shared memory, at most 220 KB.
 *                   0: the two passes below through a per-pair partial-force
 *                   buffer, shaped by [0]-[2] and [4].
 *   [0] waves       1..16: the force contraction runs over up to this many
 *                   consecutive ranges of whole structures with about equal
 *                   pair counts; the second pass of one range runs on a second
 *                   stream beside the first pass of the next, reading the
 *                   range's partial forces back from L2.
 *   [1] owner warps 4 or 8 warps per block of the first contraction pass.
 *   [2] discard     0 or 1: the second pass drops from L2 the partial-force
 *                   lines it has consumed (no write-back of dead data).
 *   [3] threads     128 or 256 threads per block of the FP32 network.
 *   [4] unroll      4, 8 or 12 partial-force slots in flight per warp in the
 *                   second contraction pass, or 16: staged in shared memory
 *                   16 slots at a time by asynchronous copies, or 1: each
 *                   atom's contiguous slot rows brought into shared memory by
 *                   bulk asynchronous copies, two pieces of up to 4 KB ahead
 *                   per warp.
 *   [6] owner_tc    0 or 1.  1 with the two passes in NEP_PREC_BF16: the
 *                   first pass on the tensor cores (tcgen05, FP16 x FP16 with
 *                   FP32 accumulation): per owner atom one MMA of its FP16
 *                   Jacobian rows (pairs, own term, virial; packed with the
 *                   dataset, each row scaled by a power of two) with its
 *                   members' FP16 input gradients; [1] does not apply.
 *                   Ignored in NEP_PREC_FP32 and by the fused form.
 *   [7] pop_pipe    0 or 1.  1 in NEP_PREC_BF16: the population network as
 *                   one persistent CTA per SM and member group, with the
 *                   bulk copies, both GEMMs and the epilogues of successive
 *                   128-atom tiles overlapped on separate warps (the same
 *                   arithmetic, the same bits).  Ignored in NEP_PREC_FP32.
 * Within each form (fused, two passes, two passes with owner_tc in BF16) no
 * shape changes a result bit (every value keeps its writer and its order of
 * summation).  The fused and two-pass forms differ in the last bits of the
 * FP32 force sums (exact in the fused form); owner_tc rounds the Jacobians
 * to FP16 (~1e-4 relative in the loss terms).
 * Default after nep_dataset_create: {1, 4, 0, 256, 4, 8, 0, 0} (members per
 * block 4, or the two passes, when the largest structure does not fit 8).
 * Errors: NEP_ERR_ARG (NULL, out of range, too little shared memory).
 */
int nep_dataset_set_shape(nep_dataset* ds, const int* shape);
int nep_dataset_get_shape(const nep_dataset* ds, int* shape);
/*
 * nep_dataset_tune -- autotuner: times every candidate shape on `reps`
 * evaluations of an n_pop-member population of fixed stand-in parameters,
 * with CUDA events on `stream` after one warm-up evaluation each, and keeps
 * the fastest on the dataset.  Candidates: the fused contraction with 4, 8
 * or 16 members per block (where the shared memory fits; the owner atoms per
 * warp are 32 / members), and the two passes with waves 1, 2, 4 x owner
 * warps 4, 8 x discard 0, 1 x unroll 1, 4, 8, 12, 16; each
 * with network threads 128, 256 in FP32 mode; in BF16 mode also every
 * two-pass candidate with owner_tc 1, and every candidate with pop_pipe 0
 * and 1.  Synchronises the stream.
 * shape_out: host int[8] or NULL; ms_out: host, the best shape's time per
 * evaluation, or NULL.
 * Errors: NEP_ERR_ARG (NULL, dataset of another model, n_pop outside 1..64,
 * reps < 1, unknown precision), NEP_ERR_OOM, NEP_ERR_CUDA.
 */
int nep_dataset_tune(nep_model* m, nep_dataset* ds, int n_pop, int precision, int reps, int* shape_out,
                     float* ms_out, void* stream);

#define NEP_PREC_FP32 0 /* network of every member in FP32 (CUDA cores) */
/* population GEMMs in BF16 with FP32 accumulation (tensor cores); the
 * two-pass contraction keeps its per-pair partial forces in FP16 (each loss
 * term averages that rounding over all force components: ~1e-6 relative) */
#define NEP_PREC_BF16 1
#define NEP_LOSS_COLS 6 /* L, L_e, L_f, L_v, L_1, L_2 */

/*
 * snes_evaluate_population -- the loss of Eq. 29 for every member of a
 * population on a training set: L = l_e L_e + l_f L_f + l_v L_v + l_1 L_1 + l_2 L_2
 * with the RMSEs of Eqs. 30-32 (energy and virial per atom) and the
 * regularisers of Eqs. 33-34.
 *   z_pop      dev [n_pop][n_par] FP32 parameter vectors, 1 <= n_pop <= 64.
 *   precision  NEP_PREC_FP32 or NEP_PREC_BF16.
 *   lambdas    host [5] = {l_e, l_f, l_v, l_1, l_2}; NULL = {1, 1, 1, 0.05, 0.05}.
 *   loss       dev [n_pop][NEP_LOSS_COLS] FP64.
 * Deterministic: fixed summation order.
 */
int snes_evaluate_population(nep_model* m, nep_dataset* ds, const float* z_pop, int n_pop, int precision,
                             const double* lambdas, double* loss, void* stream);

/*
 * nep_force_loss -- the force term of the loss for one parameter vector:
 * L_f = sqrt( sum_i |F_i - F_tar_i|^2 / (3 N) ) over the N atoms of the
 * training set (Eq. 30), with F_i from the force path (Eqs. 4-5, 23-25)
 * evaluated from the structures' positions (descriptors recomputed).
 *   z        dev [n_par] FP32 parameter vector (layout of nep_create).
 *   loss_f   dev [1] FP64, or NULL.
 * The dataset keeps a copy of z, the residuals F_i - F_tar_i and L_f, which
 * nep_force_loss_backward differentiates; one forward per backward, in
 * stream order on the same stream.  The paper fits by SNES without gradients
 * (Sec. II.D); this pair of calls is the differentiable alternative for the
 * same loss term.  Deterministic (fixed summation order).
 * Errors: NEP_ERR_ARG (NULL, dataset of another model), NEP_ERR_OOM, NEP_ERR_CUDA;
 * non-finite forces latch NEP_ERR_NONFINITE (nep_sync_status).
 */
int nep_force_loss(nep_model* m, nep_dataset* ds, const float* z, double* loss_f, void* stream);

/*
 * nep_force_loss_backward -- grad = seed * dL_f/dz at the z of the last
 * nep_force_loss on ds, by a hand-written adjoint of the force path: per atom
 * lambda_i = sum_j dq_i/dr_ij . (delta_i - delta_j), delta = (F - F_tar)/(3N L_f),
 * descriptors and their pair derivatives recomputed from the positions, then
 * the chain rule through the network of Eqs. 21-22; the sum over atoms is
 * taken in FP64 in a fixed order.  dL_f/db2 is 0; all of grad is 0 when L_f = 0.
 *   seed     dev [1] FP64 upstream gradient dOut/dL_f, or NULL for 1.
 *   grad     dev [n_par] FP64.
 * Errors: NEP_ERR_ARG (NULL, no nep_force_loss on ds before), NEP_ERR_CUDA.
 */
int nep_force_loss_backward(nep_model* m, nep_dataset* ds, const double* seed, double* grad, void* stream);

/*
 * SNES state (Sec. II.D.2, Eqs. 35-39): mean m and step sizes s (FP32,
 * n_par each), population size n_pop (2..64), and the seed of the
 * Philox4x32-10 stream that draws r_k.
 */
typedef struct snes_state snes_state;
int snes_create(nep_model* m, int n_pop, const float* mean0, const float* sigma0, unsigned long long seed,
                snes_state** out);
int snes_destroy(snes_state* st);
/*
 * snes_step -- one generation: draws r_k (standard normals, Philox4x32-10 with
 * counter {e/4, 0, generation, 0x4E4550}, Box-Muller) unless r_in (dev
 * [n_pop][n_par]) is given, forms z_k = m + s (.) r_k (Eq. 35), evaluates the
 * losses, ranks members by ascending loss (ties: lower index first), and
 * updates m then s with rank utilities u_k = max(0, ln(n/2+1) - ln k) / sum - 1/n,
 * eta_m = 1, eta_s = (3 + ln N_par) / (5 sqrt N_par) (Eqs. 36-39).
 *   loss_out   dev [n_pop][NEP_LOSS_COLS] or NULL.
 */
int snes_step(snes_state* st, nep_dataset* ds, int precision, const double* lambdas, const float* r_in,
              double* loss_out, void* stream);
/*
 * snes_run -- n_gen generations of snes_step (drawn r only), replayed from a
 * CUDA graph of one generation that is captured on the first call and kept
 * while the dataset, its launch shape, the precision and the lambdas stay the
 * same.  The generation counter of the draws lives on the device, so every
 * replay draws the next generation's numbers: the result is bit-identical to
 * n_gen calls of snes_step with r_in = NULL.
 *   n_gen      >= 0 generations.
 *   loss_hist  dev [n_gen][n_pop][NEP_LOSS_COLS] FP64 (row g: the losses of
 *              generation g of this run, unranked), or NULL.
 * Errors: NEP_ERR_ARG (NULL, dataset of another model, n_gen < 0, unknown
 * precision), NEP_ERR_OOM, NEP_ERR_CUDA (capture, instantiation or launch).
 */
int snes_run(snes_state* st, nep_dataset* ds, int precision, const double* lambdas, int n_gen, double* loss_hist,
             void* stream);
/* Copy m, s (dev [n_par]), the last draws r (dev [n_pop][n_par]) and the
 * member index at each rank (dev int [n_pop]); NULL pointers are skipped. */
int snes_get_state(snes_state* st, float* mean, float* sigma, float* r_last, int* order, void* stream);

/*
 * nep_tc_selftest -- one 128 x N x 32 BF16 tile through the tcgen05 path used
 * by NEP_PREC_BF16 (shared-memory operand layout, instruction descriptor,
 * TMEM accumulation and read-back), for checking it against a plain GEMM.
 *   A    dev, 128 x 32 BF16, row-major.
 *   B    dev, N x 32 BF16, row-major (D = A B^T); N a multiple of 16 in [16, 256].
 *   D    dev, 128 x N FP32, row-major.
 *   err  dev, 1 unsigned: error bits (8 = a bounded wait gave up), OR-ed in.
 */
int nep_tc_selftest(const void* A, const void* B, int N, float* D, unsigned* err, void* stream);

/*
 * Kernel timing: when enabled, the library records CUDA events on the
 * launching stream around each phase of its force path and integrator:
 *   NEP_PROFILE_SITE      site energies + partial forces (one kernel)
 *   NEP_PROFILE_ASSEMBLE  force / per-atom virial assembly (one kernel)
 *   NEP_PROFILE_NEIGHBOR  neighbour-list build (all its kernels; in MD they
 *                         return at once on steps without a rebuild)
 *   NEP_PROFILE_STEP      MD kick/drift, skin gate, reductions, thermo row
 * nep_profile_read synchronises, writes the summed durations (ms) and
 * bracket counts since the last read into ms[NEP_PROFILE_KINDS] and
 * launches[NEP_PROFILE_KINDS] (either may be NULL), and resets them.
 */
#define NEP_PROFILE_SITE 0
#define NEP_PROFILE_ASSEMBLE 1
#define NEP_PROFILE_NEIGHBOR 2
#define NEP_PROFILE_STEP 3
#define NEP_PROFILE_KINDS 4
int nep_profile_enable(nep_model* m, int on);
int nep_profile_read(nep_model* m, double* ms, long long* launches);

/*
 * nep_compute_efv_static -- nep_compute_efv without any device allocation.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory when they need forces -- code that runs while
 * a memory pool is locked or full by design, plugins whose host application
 * owns every allocation, or real-time loops that forbid allocator calls.  It
 * needs no model handle: the caller passes the parameters, inputs and
 * outputs, all in memory it already owns, and the scratch (neighbour list,
 * reverse index, partial forces, cells, partial sums) lives in one
 * file-scope device array of fixed size inside the library.
 *
 * Limits (the array holds about 11.6 MB on every GPU that loads the library,
 * until the process exits): n <= NEP_STATIC_MAX_ATOMS, hp->max_neighbors <=
 * NEP_STATIC_MAX_NEIGHBORS, and at most NEP_STATIC_MAX_CELLS cells of edge
 * max(rc_R, rc_A); larger inputs return NEP_ERR_ARG.  The call allocates
 * nothing: no cudaMalloc, cudaFree or allocating library routine.
 *
 * The first call in each CUDA context looks up the array's device address
 * (cudaGetSymbolAddress, with that context and its device current) and
 * caches it under the context's id; make that first call before any stream
 * capture.  A context created later (after cudaDeviceReset, or a caller's
 * own driver-API context) is a new id, so its first call looks the address
 * up again.  Every call shares the one array, which keeps
 * the previous call's contents (the parts that must start at zero are cleared
 * by the call itself); calls that overlap on the GPU -- on different streams,
 * or from host threads without ordering between them -- race on it.
 * One species only: the multicomponent weights of nep_set_species have no
 * input here, so every pair has weight 1 and n_par must be the
 * single-species count (N_des + 2) N_neu + 1.
 *   hp          host, hyperparameters as for nep_create.
 *   z           dev, n_par FP32 parameters (layout as in nep_create).
 *   n, box9, pos, e_total, e_atom, force, virial_atom, virial_total, stream:
 *               as for nep_compute_efv.
 *   err_out     dev, 1 unsigned or NULL: device-side error bits of this call
 *               (0 = none; 1 = neighbour overflow, 2 = non-finite value,
 *               4 = asymmetric list), written by the call's last kernel.
 */
#define NEP_STATIC_MAX_ATOMS 4096
#define NEP_STATIC_MAX_NEIGHBORS 96
#define NEP_STATIC_MAX_CELLS 32768
int nep_compute_efv_static(const nep_hyper* hp, const float* z, int n_par, int n, const double* box9,
                           const double* pos, double* e_total, double* e_atom, float* force, float* virial_atom,
                           double* virial_total, unsigned* err_out, void* stream);

/* Message describing the last failing call on this thread ("" if none). */
const char* nep_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* NEP_H */
