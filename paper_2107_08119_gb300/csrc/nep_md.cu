// nep_md.cu -- NVE velocity-Verlet molecular dynamics on the NEP force path.
//
// One step is a fixed sequence of kernels on the caller's stream, with no
// host round trip:
//   k_kick_drift   v += dt/2 F/m; x += dt v (FP64); FP32 hi/lo split of x;
//                  largest squared displacement since the last list build
//   k_decide       gate = (max displacement > skin/2) or a pending rebuild
//   list build     wrap, bin, Verlet list, reverse index (gated: the kernels
//                  return at once when the gate is zero)
//   k_site         site energies and partial forces
//   k_assemble     forces, second half kick, E_kin, virial and heat current
//                  J = sum_i W_i . v_i (Eq. 7), per-block FP64 sums
//   k_md_finish    block sums in a fixed order, thermo row and J of this
//                  step, Berendsen factor
// Optional extensions (nep_md_set_thermostat, nep_md_set_hnemd):
//   HNEMD          the assembly writes F and W_i; after the virial sum,
//                  k_hnemd_kick adds F_i^ext = F_e . W_i - F_e . W / N
//                  (Sec. II.B; the mean removed so the momentum is kept) and
//                  does the second half kick, E_kin and J
//   thermostat     Berendsen: after J, v *= lambda with lambda^2 = 1 +
//                  (dt/tau)(T0/T - 1), T from E_kin with 3N - 3 degrees of
//                  freedom (k_scale_v)
#include <cmath>
#include <new>

#include "nep_internal.cuh"

// 1 amu A^2 / fs^2 expressed in eV (CODATA 2018 atomic mass constant and
// elementary charge).
static constexpr double kAmuA2Fs2InEv = 1.66053906660e-27 * 1.0e-20 / 1.0e-30 / 1.602176634e-19;
// Boltzmann constant in eV/K (CODATA 2018)
static constexpr double kBoltzmannEv = 8.617333262e-5;

namespace nep {
namespace {

// control words on the device
enum { kCtlDisp = 0, kCtlGate = 1, kCtlPending = 2, kCtlStep = 3, kCtlWords = 4 };

__global__ void k_kick_drift(int n, double* __restrict__ x, double* __restrict__ v, const float* __restrict__ F,
                             double hdtm, double dt, float* __restrict__ xh, float* __restrict__ xl,
                             const double* __restrict__ x_ref, unsigned* __restrict__ ctl)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float d2 = 0.f;
    if (i < n) {
        double dd = 0.0, xn[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t o = (size_t)c * n + i;
            const double vc = v[o] + hdtm * (double)F[o];
            const double xc = x[o] + dt * vc;
            v[o] = vc;
            x[o] = xc;
            xn[c] = xc;
            const double d = xc - x_ref[o];
            dd += d * d;
        }
        store_pos(xh, xl, i, xn);
        d2 = (float)dd;
    }
    // block maximum, then one atomic per block (one per warp serialised
    // thousands of atomics on a single word)
    __shared__ float wmax[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d2 = fmaxf(d2, __shfl_xor_sync(0xffffffffu, d2, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = d2;
    __syncthreads();
    if (threadIdx.x < 32) {
        d2 = threadIdx.x < (blockDim.x >> 5) ? wmax[threadIdx.x] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d2 = fmaxf(d2, __shfl_xor_sync(0xffffffffu, d2, o));
        // non-negative floats order like their bit patterns
        if (threadIdx.x == 0 && d2 > 0.f) atomicMax(ctl + kCtlDisp, __float_as_uint(d2));
    }
}

__global__ void k_decide(unsigned* __restrict__ ctl, float thresh2, unsigned long long* __restrict__ rebuilds)
{
    const bool go = ctl[kCtlPending] != 0u || __uint_as_float(ctl[kCtlDisp]) > thresh2;
    ctl[kCtlGate] = go ? 1u : 0u;
    ctl[kCtlDisp] = 0u;
    ctl[kCtlPending] = 0u;
    if (go) *rebuilds += 1ull;
}

// Second half kick with the HNEMD driving force, E_kin and J per block.
// W is the per-atom virial [9][n]; wtot the total virial (row-major).
__global__ void k_hnemd_kick(int n, float* __restrict__ F, const float* __restrict__ W, double* __restrict__ vel,
                             double fe0, double fe1, double fe2, const double* __restrict__ wtot, double inv_n,
                             double hdtm, double kef, double* __restrict__ partials, unsigned* err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (i < n) {
        const double fe[3] = {fe0, fe1, fe2};
        float w[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) w[c] = W[(size_t)c * n + i];
        double v[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            double fx = 0.0, fm = 0.0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                fx += fe[a] * (double)w[3 * a + b];
                fm += fe[a] * wtot[3 * a + b];
            }
            const float ft = (float)((double)F[(size_t)b * n + i] + fx - fm * inv_n);
            F[(size_t)b * n + i] = ft;
            v[b] = vel[(size_t)b * n + i] + hdtm * (double)ft;
            vel[(size_t)b * n + i] = v[b];
        }
        if (!isfinite(v[0] + v[1] + v[2])) atomicOr(err, kErrNonFinite);
        acc[0] = kef * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
#pragma unroll
        for (int a = 0; a < 3; ++a)
            acc[1 + a] = (double)(w[3 * a] * (float)v[0]) + (double)(w[3 * a + 1] * (float)v[1]) +
                         (double)(w[3 * a + 2] * (float)v[2]);
    }
    block_sum_store<4>(acc, partials + (size_t)blockIdx.x * 4);
}

// v *= lambda (the Berendsen factor k_md_finish left in red[14])
__global__ void k_scale_v(int n, double* __restrict__ vel, const double* __restrict__ red)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double lam = red[14];
#pragma unroll
    for (int c = 0; c < 3; ++c) vel[(size_t)c * n + i] *= lam;
}

// The step's last kernel: warp 0 sums the site-energy block partials into
// red[0], warp 1 + c sums component c of the other block partials into
// red[off_x + c] (fixed order, like k_reduce), then thread 0 writes the thermo
// row and J and the Berendsen factor.
__global__ void k_md_finish(const double* __restrict__ part_e, int nb_e, const double* __restrict__ part_x, int nb_x,
                            int ncomp_x, int off_x, double* __restrict__ red, double* __restrict__ thermo,
                            double* __restrict__ heat, unsigned* __restrict__ ctl, double t0, double tau, double dt,
                            double dof_kb)
{
    // red: [0] E_pot, [1..9] W (row-major), [10] E_kin, [11..13] J, [14] lambda
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w <= ncomp_x) {
        const double* src = w == 0 ? part_e : part_x + (w - 1);
        const int nb = w == 0 ? nb_e : nb_x;
        const int stride = w == 0 ? 1 : ncomp_x;
        double v = 0.0;
        for (int b = lane; b < nb; b += 32) v += src[(size_t)b * stride];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[w == 0 ? 0 : off_x + w - 1] = v;
    }
    __syncthreads();
    const unsigned s = ctl[kCtlStep];
    if (threadIdx.x == 0) {
        double ek = red[10];
        if (tau > 0.0) {
            const double T = 2.0 * ek / dof_kb;
            const double lam = T > 0.0 ? sqrt(1.0 + dt / tau * (t0 / T - 1.0)) : 1.0;
            red[14] = lam;
            ek *= lam * lam;
        }
        if (thermo) {
            double* t = thermo + (size_t)s * NEP_THERMO_COLS;
            t[0] = red[0];
            t[1] = ek;
            t[2] = red[1];  // xx
            t[3] = red[5];  // yy
            t[4] = red[9];  // zz
            t[5] = red[2];  // xy
            t[6] = red[6];  // yz
            t[7] = red[7];  // zx
        }
        if (heat) {
            heat[(size_t)s * 3 + 0] = red[11];
            heat[(size_t)s * 3 + 1] = red[12];
            heat[(size_t)s * 3 + 2] = red[13];
        }
        ctl[kCtlStep] = s + 1u;
    }
}

inline int blocks_for(int n, int t) { return (n + t - 1) / t; }

}  // namespace
}  // namespace nep

using namespace nep;

struct nep_md {
    nep_model* m = nullptr;
    int n = 0;
    Box box;
    double mass = 0.0;
    float r_list = 0.f;
    float skin = 0.f;
    Workspace ws;
    double* x_ref = nullptr;
    unsigned* ctl = nullptr;
    unsigned long long* rebuilds = nullptr;
    double* red = nullptr;
    bool need_init = true;
    // Berendsen thermostat (tau <= 0: off) and HNEMD driving force
    double t0 = 0.0, tau = 0.0;
    double fe[3] = {0.0, 0.0, 0.0};
    bool drive = false;
    float* w_atom = nullptr;  // [9][n] per-atom virials (HNEMD only)
};

extern "C" {

int nep_md_create(nep_model* m, int n, const double* box9, double mass, nep_md** out)
{
    if (!m || !out || n < 1 || n > kMaxAtoms || !(mass > 0.0)) {
        set_error("nep_md_create: bad arguments");
        return NEP_ERR_ARG;
    }
    *out = nullptr;
    const double rmax = (m->hp.rc_R > m->hp.rc_A ? m->hp.rc_R : m->hp.rc_A) + m->hp.skin;
    nep_md* md = new (std::nothrow) nep_md();
    if (!md) {
        set_error("nep_md_create: host allocation failed");
        return NEP_ERR_OOM;
    }
    int rc = setup_box(box9, rmax, md->box);
    if (rc) {
        delete md;
        return rc;
    }
    md->m = m;
    md->n = n;
    md->mass = mass;
    md->r_list = (float)rmax;
    md->skin = (float)m->hp.skin;
    const int ncell = md->box.nc[0] * md->box.nc[1] * md->box.nc[2];
    const int nb = site_blocks(n);
    if ((rc = ensure_workspace(md->ws, n, m->hp.max_neighbors, ncell, nb))) {
        nep_md_destroy(md);
        return rc;
    }
    cudaError_t e = cudaMalloc((void**)&md->x_ref, sizeof(double) * 3 * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&md->ctl, sizeof(unsigned) * kCtlWords);
    if (e == cudaSuccess) e = cudaMalloc((void**)&md->rebuilds, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc((void**)&md->red, sizeof(double) * 32);
    if (e == cudaSuccess) e = cudaMemset(md->ctl, 0, sizeof(unsigned) * kCtlWords);
    if (e == cudaSuccess) e = cudaMemset(md->rebuilds, 0, sizeof(unsigned long long));
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("nep_md_create: %s", cudaGetErrorString(e));
        nep_md_destroy(md);
        return NEP_ERR_OOM;
    }
    *out = md;
    return NEP_OK;
}

int nep_md_destroy(nep_md* md)
{
    if (!md) return NEP_OK;
    cudaDeviceSynchronize();
    free_workspace(md->ws);
    if (md->x_ref) cudaFree(md->x_ref);
    if (md->ctl) cudaFree(md->ctl);
    if (md->rebuilds) cudaFree(md->rebuilds);
    if (md->red) cudaFree(md->red);
    if (md->w_atom) cudaFree(md->w_atom);
    delete md;
    return NEP_OK;
}

int nep_md_set_thermostat(nep_md* md, double t0, double tau)
{
    if (!md || (tau > 0.0 && !(t0 >= 0.0))) {
        set_error("nep_md_set_thermostat: NULL handle or negative target temperature");
        return NEP_ERR_ARG;
    }
    md->t0 = t0;
    md->tau = tau > 0.0 ? tau : 0.0;
    return NEP_OK;
}

int nep_md_set_hnemd(nep_md* md, const double* fe)
{
    if (!md) {
        set_error("nep_md_set_hnemd: NULL handle");
        return NEP_ERR_ARG;
    }
    for (int c = 0; c < 3; ++c) md->fe[c] = fe ? fe[c] : 0.0;
    md->drive = md->fe[0] != 0.0 || md->fe[1] != 0.0 || md->fe[2] != 0.0;
    if (md->drive && !md->w_atom) {
        cudaError_t e = cudaMalloc((void**)&md->w_atom, sizeof(float) * 9 * (size_t)md->n);
        if (e != cudaSuccess) {
            cudaGetLastError();
            md->w_atom = nullptr;
            md->drive = false;
            set_error("nep_md_set_hnemd: %s", cudaGetErrorString(e));
            return NEP_ERR_OOM;
        }
    }
    md->need_init = true;  // the next step recomputes the starting forces with (or without) the drive
    return NEP_OK;
}

int nep_md_invalidate(nep_md* md)
{
    if (!md) {
        set_error("nep_md_invalidate: NULL handle");
        return NEP_ERR_ARG;
    }
    md->need_init = true;
    return NEP_OK;
}

int nep_md_rebuild_count(nep_md* md, long long* count, void* stream)
{
    if (!md || !count) {
        set_error("nep_md_rebuild_count: NULL argument");
        return NEP_ERR_ARG;
    }
    int rc = cuda_fail(cudaStreamSynchronize((cudaStream_t)stream), "stream synchronise");
    if (rc) return rc;
    unsigned long long c = 0;
    rc = cuda_fail(cudaMemcpy(&c, md->rebuilds, sizeof(c), cudaMemcpyDeviceToHost), "read rebuild count");
    *count = (long long)c;
    return rc;
}

const float* nep_md_forces(const nep_md* md) { return md ? md->ws.force : nullptr; }

int nep_md_step(nep_md* md, double* pos, double* vel, int n_steps, double dt, double* thermo, double* heat,
                void* stream)
{
    if (!md || !pos || !vel || n_steps < 0 || !(dt > 0.0)) {
        set_error("nep_md_step: bad arguments");
        return NEP_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    nep_model* m = md->m;
    const int n = md->n;
    NeighborList& nl = md->ws.nl;
    const int nb = site_blocks(n);
    double* part_e = md->ws.partials;
    double* part_a = md->ws.partials + ((nb + 7) / 8) * 8;
    double* part_h = part_a + 13 * (size_t)blocks_for(n, 128);  // HNEMD kick partials
    const bool drive = md->drive;
    const int nbk = blocks_for(n, 256);
    const double kef = 0.5 * md->mass * kAmuA2Fs2InEv;
    ForceArgs fa{m->d_z, m->hp.n_neu, (float)m->hp.rc_R, (float)m->hp.rc_A, md->box};
    const double rmax = m->hp.rc_R > m->hp.rc_A ? m->hp.rc_R : m->hp.rc_A;
    const double conv = kAmuA2Fs2InEv;
    int rc;
    const unsigned* gate = md->ctl + kCtlGate;
    if (md->tau > 0.0 && n < 2) {
        set_error("nep_md_step: the thermostat needs at least two atoms");
        return NEP_ERR_ARG;
    }

    if (md->need_init) {
        // forces of the starting configuration (list built unconditionally)
        if ((rc = build_neighbor_list(nl, md->box, n, pos, true, md->x_ref, md->r_list, m->d_err, nullptr, st)))
            return rc;
        int b1 = 0, b2 = 0, c2 = 0;
        if ((rc = launch_site_partial_forces(fa, nl, n, nullptr, part_e, m->d_err, st, b1))) return rc;
        AssembleArgs aa{};
        aa.rc_max = (float)rmax;
        aa.box = md->box;
        aa.vel = nullptr;
        if ((rc = launch_assemble(aa, nl, n, md->ws.force, drive ? md->w_atom : nullptr, part_a, m->d_err, st, b2,
                                  c2)))
            return rc;
        if (drive) {
            // the starting forces include the driving force (no kick: hdt/m = 0)
            if ((rc = launch_reduce(part_a, b2, c2, md->red + 1, st))) return rc;
            k_hnemd_kick<<<nbk, 256, 0, st>>>(n, md->ws.force, md->w_atom, vel, md->fe[0], md->fe[1], md->fe[2],
                                              md->red + 1, 1.0 / n, 0.0, kef, part_h, m->d_err);
        }
        if ((rc = cuda_fail(cudaMemsetAsync(md->ctl, 0, sizeof(unsigned) * kCtlWords, st), "cudaMemsetAsync")))
            return rc;
        md->need_init = false;
    }
    if ((rc = cuda_fail(cudaMemsetAsync(md->ctl + kCtlStep, 0, sizeof(unsigned), st), "cudaMemsetAsync"))) return rc;

    const double hdtm = 0.5 * dt / (md->mass * conv);
    const float thresh = 0.5f * md->skin;
    for (int s = 0; s < n_steps; ++s) {
        Profiler::Slot* pk = m->prof.begin(NEP_PROFILE_STEP, st);
        k_kick_drift<<<blocks_for(n, 256), 256, 0, st>>>(n, pos, vel, md->ws.force, hdtm, dt, nl.xh, nl.xl, md->x_ref,
                                                         md->ctl);
        k_decide<<<1, 1, 0, st>>>(md->ctl, thresh * thresh, md->rebuilds);
        m->prof.end(pk, st);
        pk = m->prof.begin(NEP_PROFILE_NEIGHBOR, st);
        if ((rc = build_neighbor_list(nl, md->box, n, pos, true, md->x_ref, md->r_list, m->d_err, gate, st)))
            return rc;
        m->prof.end(pk, st);
        int b1 = 0, b2 = 0, c2 = 0;
        Profiler::Slot* ps = m->prof.begin(NEP_PROFILE_SITE, st);
        if ((rc = launch_site_partial_forces(fa, nl, n, nullptr, part_e, m->d_err, st, b1))) return rc;
        m->prof.end(ps, st);
        AssembleArgs aa{};
        aa.rc_max = (float)rmax;
        aa.box = md->box;
        aa.vel = drive ? nullptr : vel;  // with HNEMD the kick waits for the total virial
        aa.half_dt_over_m = hdtm;
        aa.ke_factor = kef;
        aa.heat = heat != nullptr;
        ps = m->prof.begin(NEP_PROFILE_ASSEMBLE, st);
        if ((rc = launch_assemble(aa, nl, n, md->ws.force, drive ? md->w_atom : nullptr, part_a, m->d_err, st, b2,
                                  c2)))
            return rc;
        m->prof.end(ps, st);
        pk = m->prof.begin(NEP_PROFILE_STEP, st);
        const double dof_kb = (3.0 * n - 3.0) * kBoltzmannEv;
        if (drive) {
            // the kick needs the total virial first
            if ((rc = launch_reduce(part_a, b2, c2, md->red + 1, st))) return rc;
            k_hnemd_kick<<<nbk, 256, 0, st>>>(n, md->ws.force, md->w_atom, vel, md->fe[0], md->fe[1], md->fe[2],
                                              md->red + 1, 1.0 / n, hdtm, kef, part_h, m->d_err);
            k_md_finish<<<1, 32 * 5, 0, st>>>(part_e, b1, part_h, nbk, 4, 10, md->red, thermo, heat, md->ctl, md->t0,
                                              md->tau, dt, dof_kb);
        } else {
            k_md_finish<<<1, 32 * (1 + c2), 0, st>>>(part_e, b1, part_a, b2, c2, 1, md->red, thermo, heat, md->ctl,
                                                     md->t0, md->tau, dt, dof_kb);
        }
        if (md->tau > 0.0 && n > 1) k_scale_v<<<nbk, 256, 0, st>>>(n, vel, md->red);
        m->prof.end(pk, st);
        if ((rc = cuda_fail(cudaGetLastError(), "md step kernels"))) return rc;
    }
    return NEP_OK;
}

}  // extern "C"
