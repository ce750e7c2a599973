// nep_md.cu -- NVE velocity-Verlet molecular dynamics on the NEP force path.
//
// One step is a fixed sequence of kernels on the caller's stream, with no
// host round trip:
//   k_kick_drift   v += dt/2 F/m; x += dt v (FP64); FP32 hi/lo split of x;
//                  largest squared displacement since the last list build;
//                  its last block sets the gate = (max displacement >
//                  skin/2) or a pending rebuild
//   list build     wrap, bin, Verlet list, reverse index (gated: the kernels
//                  return at once when the gate is zero)
//   k_site         site energies and partial forces
//   k_assemble     forces, second half kick, E_kin, virial and heat current
//                  J = sum_i W_i . v_i (Eq. 7), per-block FP64 sums
//   k_md_finish    block sums in a fixed order (one block per sum), thermo
//                  row and J of this step, Berendsen factor
// Optional extensions (nep_md_set_thermostat, nep_md_set_hnemd):
//   HNEMD          the assembly writes F and W_i; after the virial sum,
//                  k_hnemd_kick adds F_i^ext = F_e . W_i - F_e . W / N
//                  (Sec. II.B; the mean removed so the momentum is kept) and
//                  does the second half kick, E_kin and J
//   thermostat     Berendsen: after J, v *= lambda with lambda^2 = 1 +
//                  (dt/tau)(T0/T - 1), T from E_kin with 3N - 3 degrees of
//                  freedom (k_scale_v)
//   spectral heat current (nep_md_set_shc): on every `every`-th step the
//                  assembly writes W_i into a ring of n_lags samples and,
//                  next to J, k_shc_corr / k_shc_reduce add
//                  sum_i W_i(s - tau) . v_i(s) to K[tau] for every lag tau
//                  already in the ring (Sec. II.B)
#include <cmath>
#include <new>

#include "nep_internal.cuh"

// 1 amu A^2 / fs^2 expressed in eV (CODATA 2018 atomic mass constant and
// elementary charge).
static constexpr double kAmuA2Fs2InEv = 1.66053906660e-27 * 1.0e-20 / 1.0e-30 / 1.602176634e-19;
// Boltzmann constant in eV/K (CODATA 2018)
static constexpr double kBoltzmannEv = 8.617333262e-5;
// reduced Planck constant in eV fs (CODATA 2018)
static constexpr double kHbarEvFs = 0.6582119569;
static constexpr double kPi = 3.14159265358979323846;
// 1 eV / (A fs K) in W / (m K): 1.602176634e-19 J / (1e-10 m 1e-15 s K)
static constexpr double kEvPerAFsK_WPerMK = 1.602176634e6;

namespace nep {
namespace {

// control words on the device
enum { kCtlDisp = 0, kCtlGate = 1, kCtlPending = 2, kCtlStep = 3, kCtlFinish = 4, kCtlKick = 5, kCtlWords = 6 };

// The rebuild decision: gate = a pending rebuild or the largest squared
// displacement since the last build above thresh2; the displacement and the
// pending flag are cleared.  use_cond: the step runs from a CUDA graph whose
// list rebuild sits behind the conditional node `cond`, which this sets.
__device__ void decide(unsigned* ctl, float thresh2, unsigned long long* rebuilds, cudaGraphConditionalHandle cond,
                       int use_cond)
{
    const unsigned disp = __ldcg(ctl + kCtlDisp);
    const bool go = __ldcg(ctl + kCtlPending) != 0u || __uint_as_float(disp) > thresh2;
    ctl[kCtlGate] = go ? 1u : 0u;
    ctl[kCtlDisp] = 0u;
    ctl[kCtlPending] = 0u;
    if (go) *rebuilds += 1ull;
    if (use_cond) cudaGraphSetConditional(cond, go ? 1u : 0u);
}

__global__ void k_kick_drift(int n, double* __restrict__ x, double* __restrict__ v, const float* __restrict__ F,
                             double hdtm, double dt, float* __restrict__ xh, float* __restrict__ xl,
                             const double* __restrict__ x_ref, unsigned* __restrict__ ctl, float thresh2,
                             unsigned long long* __restrict__ rebuilds, cudaGraphConditionalHandle cond, int use_cond)
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
        store_pos(xh, xl, i, xn, load_z(xh, i));  // the species number stays
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
    // the last block to finish (a count in ctl, which it clears) takes the
    // rebuild decision
    __shared__ int last;
    if (threadIdx.x == 0) {
        __threadfence();  // this block's maximum before the count
        last = atomicAdd(ctl + kCtlKick, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    ctl[kCtlKick] = 0u;
    decide(ctl, thresh2, rebuilds, cond, use_cond);
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

// Virial-velocity correlation of one sample s (the ring holds W of the last
// `avail` samples, sample s in slot `slot0`): warp w of block (bx, by) takes
// lag tau = 8 bx + w and the atoms of chunk by, and writes
// sum_i (W_i(s - tau) . v_i(s))^a for its chunk, in a fixed order (lane
// strides, then a butterfly), to part[by][tau][a].  The products are FP32
// and the sums FP64, as in the heat current of the assembly.
constexpr int kShcChunk = 4096;
constexpr int kShcLagsPerBlock = 8;

__global__ void __launch_bounds__(32 * kShcLagsPerBlock) k_shc_corr(int n, int n_lags, int avail, int slot0,
                                                                      const float* __restrict__ ring,
                                                                      const double* __restrict__ vel,
                                                                      double* __restrict__ part)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tau = blockIdx.x * kShcLagsPerBlock + warp;
    if (tau >= avail) return;  // warp-uniform
    const int slot = (slot0 - tau + n_lags) % n_lags;
    const float* W = ring + (size_t)slot * 9 * n;
    const int c0 = blockIdx.y * kShcChunk, c1 = min(n, c0 + kShcChunk);
    double acc[3] = {0.0, 0.0, 0.0};
    for (int i = c0 + lane; i < c1; i += 32) {
        const float v0 = (float)vel[i], v1 = (float)vel[(size_t)n + i], v2 = (float)vel[2 * (size_t)n + i];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            acc[a] += (double)(W[(size_t)(3 * a) * n + i] * v0) + (double)(W[(size_t)(3 * a + 1) * n + i] * v1) +
                      (double)(W[(size_t)(3 * a + 2) * n + i] * v2);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], o);
    if (lane == 0)
#pragma unroll
        for (int a = 0; a < 3; ++a) part[((size_t)blockIdx.y * n_lags + tau) * 3 + a] = acc[a];
}

// sum[tau][a] += the chunk partials of this sample, chunks in order
__global__ void k_shc_reduce(int n_lags, int avail, int n_chunks, const double* __restrict__ part,
                             double* __restrict__ sum)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= avail * 3) return;
    const int tau = e / 3, a = e % 3;
    double t = 0.0;
    for (int c = 0; c < n_chunks; ++c) t += part[((size_t)c * n_lags + tau) * 3 + a];
    sum[(size_t)tau * 3 + a] += t;
}

// K[tau] = sum[tau] / (number of origins), 0 without any
__global__ void k_shc_average(int n_lags, long long n_samples, const double* __restrict__ sum, double* __restrict__ K)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_lags * 3) return;
    const long long origins = n_samples - e / 3;
    K[e] = origins > 0 ? sum[e] / (double)origins : 0.0;
}

// out[k][a] = scale * 2 * trapezoid of K[tau][a] cos(omega_k tau dt) over the
// lags (K even in t), optionally Hann-windowed (Sec. II.B transform)
// omega_k = omega_per_x * x[k] (1 when x holds the angular frequencies).
__global__ void k_shc_spectrum(int n_lags, const double* __restrict__ K, double dt, int n_omega,
                               const double* __restrict__ omega, double omega_per_x, double scale, int window,
                               double* __restrict__ out)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_omega * 3) return;
    const int k = e / 3, a = e % 3;
    const double w0 = omega_per_x * omega[k];
    double s = 0.0;
    for (int t = 0; t < n_lags; ++t) {
        double w = (t == 0 || t == n_lags - 1) ? 0.5 : 1.0;
        if (window && n_lags > 1) w *= 0.5 * (1.0 + cospi((double)t / (n_lags - 1)));
        s += w * K[(size_t)t * 3 + a] * cos(w0 * t * dt);
    }
    out[e] = scale * 2.0 * dt * s;
}

// spec[k][.] *= (h / sinh h)^2 with h = x/2, x = x_per_omega omega[k]: the
// quantum-correction factor x^2 e^x / (e^x - 1)^2 of Sec. IV.C in a form with
// no cancellation at small x (1 - h^2/3 below h = 1e-4, where FP64 sinh(h)/h
// has nothing left to resolve) and none at large x (sinh overflows to inf and
// the factor to 0).
__global__ void k_shc_quantum(int n_omega, const double* __restrict__ omega, double x_per_omega,
                              double* __restrict__ spec)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_omega) return;
    const double h = fabs(0.5 * (x_per_omega * omega[k]));
    double f;
    if (h < 1e-4) {
        f = 1.0 - h * h / 3.0;
    } else {
        const double r = h / sinh(h);
        f = r * r;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) spec[(size_t)k * 3 + a] *= f;
}

// Running mean of J times scale: thread t of one block owns a contiguous
// segment of steps; the segment sums are prefixed in order by thread 0, and
// each thread then walks its segment again from its offset.
constexpr int kKappaThreads = 256;
__global__ void __launch_bounds__(kKappaThreads) k_hnemd_kappa(int n, const double* __restrict__ J, double scale,
                                                               double* __restrict__ out)
{
    __shared__ double seg[kKappaThreads][3];
    const int t = threadIdx.x;
    const int per = (n + kKappaThreads - 1) / kKappaThreads;
    const int a = min(n, t * per), b = min(n, a + per);
    double s[3] = {0.0, 0.0, 0.0};
    for (int i = a; i < b; ++i)
#pragma unroll
        for (int c = 0; c < 3; ++c) s[c] += J[(size_t)i * 3 + c];
#pragma unroll
    for (int c = 0; c < 3; ++c) seg[t][c] = s[c];
    __syncthreads();
    if (t == 0) {
        double run[3] = {0.0, 0.0, 0.0};
        for (int u = 0; u < kKappaThreads; ++u)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double x = seg[u][c];
                seg[u][c] = run[c];
                run[c] += x;
            }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 3; ++c) s[c] = seg[t][c];
    for (int i = a; i < b; ++i)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            s[c] += J[(size_t)i * 3 + c];
            out[(size_t)i * 3 + c] = scale * s[c] / (double)(i + 1);
        }
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

// The step's last kernel, one block per sum: block 0 adds the site-energy
// block partials into red[0], block 1 + c component c of the other block
// partials into red[off_x + c] (each thread a fixed stride of the partials in
// order, then a fixed tree: deterministic).  Several SMs share the FP64 adds
// (slow on this part).  The last block to finish (a count in ctl, which it
// clears) writes the thermo row and J and the Berendsen factor.
constexpr int kFinishThreads = 128;

__global__ void __launch_bounds__(kFinishThreads) k_md_finish(const double* __restrict__ part_e, int nb_e,
                                                              const double* __restrict__ part_x, int nb_x,
                                                              int ncomp_x, int off_x, double* __restrict__ red,
                                                              double* __restrict__ thermo, double* __restrict__ heat,
                                                              unsigned* __restrict__ ctl, double t0, double tau,
                                                              double dt, double dof_kb)
{
    // red: [0] E_pot, [1..9] W (row-major), [10] E_kin, [11..13] J, [14] lambda
    const int w = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double* src = w == 0 ? part_e : part_x + (w - 1);
    const int nb = w == 0 ? nb_e : nb_x;
    const int stride = w == 0 ? 1 : ncomp_x;
    double v = 0.0;
    // unrolled so that eight loads are in flight ahead of the (ordered) adds
#pragma unroll 8
    for (int b = threadIdx.x; b < nb; b += kFinishThreads) v += src[(size_t)b * stride];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __shared__ double wsum[kFinishThreads / 32];
    __shared__ int last;
    if (lane == 0) wsum[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < kFinishThreads / 32; ++q) t += wsum[q];
        red[w == 0 ? 0 : off_x + w - 1] = t;
        __threadfence();  // this sum before the count
        last = atomicAdd(ctl + kCtlFinish, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    ctl[kCtlFinish] = 0u;
    // the other blocks' sums, read from L2
    auto rd = [&](int k) { return __ldcg(red + k); };
    const unsigned s = ctl[kCtlStep];
    double ek = rd(10);
    if (tau > 0.0) {
        const double T = 2.0 * ek / dof_kb;
        const double lam = T > 0.0 ? sqrt(1.0 + dt / tau * (t0 / T - 1.0)) : 1.0;
        red[14] = lam;
        ek *= lam * lam;
    }
    if (thermo) {
        double* t = thermo + (size_t)s * NEP_THERMO_COLS;
        t[0] = rd(0);
        t[1] = ek;
        t[2] = rd(1);  // xx
        t[3] = rd(5);  // yy
        t[4] = rd(9);  // zz
        t[5] = rd(2);  // xy
        t[6] = rd(6);  // yz
        t[7] = rd(7);  // zx
    }
    if (heat) {
        heat[(size_t)s * 3 + 0] = rd(11);
        heat[(size_t)s * 3 + 1] = rd(12);
        heat[(size_t)s * 3 + 2] = rd(13);
    }
    ctl[kCtlStep] = s + 1u;
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
    bool plain = false;       // force pass by the plain FP32 comparator (nep_md_set_force_form)
    float* w_atom = nullptr;  // [9][n] per-atom virials (HNEMD only)
    // spectral heat current: ring of per-atom virials, lag sums, chunk partials
    int shc_lags = 0, shc_every = 1;
    long long shc_step = 0, shc_samples = 0;
    float* shc_ring = nullptr;   // [n_lags][9][n]
    double* shc_sum = nullptr;   // [n_lags][3]
    double* shc_part = nullptr;  // [chunks][n_lags][3]
    // one step captured as a CUDA graph (the list rebuild behind a conditional
    // node), kept while everything it bakes in is unchanged
    cudaStream_t gcap = nullptr, gcap2 = nullptr;
    cudaGraphExec_t gexec = nullptr;
    struct GraphKey {
        const double *pos, *vel;
        double *thermo, *heat;
        double dt, t0, tau, fe[3];
        bool drive;
        const float* zatom;
        bool plain;
        bool operator==(const GraphKey& o) const
        {
            return pos == o.pos && vel == o.vel && thermo == o.thermo && heat == o.heat && dt == o.dt &&
                   t0 == o.t0 && tau == o.tau && fe[0] == o.fe[0] && fe[1] == o.fe[1] && fe[2] == o.fe[2] &&
                   drive == o.drive && zatom == o.zatom && plain == o.plain;
        }
    } gkey{};
};

namespace {
// the model's species numbers when they were set for this many atoms
const float* md_zatom(const nep_md* md)
{
    return md->m->zatom && md->m->zatom_n == md->n ? md->m->zatom : nullptr;
}

void free_shc(nep_md* md)
{
    if (md->shc_ring) cudaFree(md->shc_ring);
    if (md->shc_sum) cudaFree(md->shc_sum);
    if (md->shc_part) cudaFree(md->shc_part);
    md->shc_ring = nullptr;
    md->shc_sum = nullptr;
    md->shc_part = nullptr;
    md->shc_lags = 0;
    md->shc_step = md->shc_samples = 0;
}
}  // namespace

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
    free_shc(md);
    if (md->gexec) cudaGraphExecDestroy(md->gexec);
    if (md->gcap) cudaStreamDestroy(md->gcap);
    if (md->gcap2) cudaStreamDestroy(md->gcap2);
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

int nep_md_set_force_form(nep_md* md, int form)
{
    if (!md || (form != NEP_FORCE_OPTIMISED && form != NEP_FORCE_PLAIN_FP32)) {
        set_error("nep_md_set_force_form: NULL handle or unknown form %d", form);
        return NEP_ERR_ARG;
    }
    if (form == NEP_FORCE_PLAIN_FP32 && !sizes_default(md->m->hp)) {
        set_error("nep_md_set_force_form: the plain comparator has kernels for the 32-descriptor model only");
        return NEP_ERR_UNSUPPORTED;
    }
    if (form == NEP_FORCE_PLAIN_FP32 && md->ws.plain_cap < md->n) {
        if (md->ws.plain) cudaFree(md->ws.plain);
        md->ws.plain = nullptr;
        md->ws.plain_cap = 0;
        const cudaError_t e = cudaMalloc((void**)&md->ws.plain, sizeof(float) * 2 * kNdes * (size_t)md->n);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("nep_md_set_force_form: %s", cudaGetErrorString(e));
            return NEP_ERR_OOM;
        }
        md->ws.plain_cap = md->n;
    }
    md->plain = form == NEP_FORCE_PLAIN_FP32;
    md->need_init = true;  // the next step recomputes the starting forces with the selected form
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

int nep_md_set_shc(nep_md* md, int n_lags, int every)
{
    if (!md || n_lags < 0 || n_lags > 100000 || (n_lags > 0 && every < 1)) {
        set_error("nep_md_set_shc: bad arguments (0 <= n_lags <= 100000, every >= 1)");
        return NEP_ERR_ARG;
    }
    cudaDeviceSynchronize();
    free_shc(md);
    if (n_lags == 0) return NEP_OK;
    const int chunks = (md->n + kShcChunk - 1) / kShcChunk;
    cudaError_t e = cudaMalloc((void**)&md->shc_ring, sizeof(float) * 9 * (size_t)md->n * n_lags);
    if (e == cudaSuccess) e = cudaMalloc((void**)&md->shc_sum, sizeof(double) * 3 * (size_t)n_lags);
    if (e == cudaSuccess) e = cudaMalloc((void**)&md->shc_part, sizeof(double) * 3 * (size_t)n_lags * chunks);
    if (e == cudaSuccess) e = cudaMemset(md->shc_sum, 0, sizeof(double) * 3 * (size_t)n_lags);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_shc(md);
        set_error("nep_md_set_shc: %s", cudaGetErrorString(e));
        return NEP_ERR_OOM;
    }
    md->shc_lags = n_lags;
    md->shc_every = every;
    return NEP_OK;
}

int nep_md_get_shc(nep_md* md, double* K, long long* n_samples, void* stream)
{
    if (!md || md->shc_lags == 0) {
        set_error("nep_md_get_shc: NULL handle or no correlation switched on (nep_md_set_shc)");
        return NEP_ERR_ARG;
    }
    if (n_samples) *n_samples = md->shc_samples;
    if (K) {
        const int e = md->shc_lags * 3;
        k_shc_average<<<(e + 255) / 256, 256, 0, (cudaStream_t)stream>>>(md->shc_lags, md->shc_samples, md->shc_sum,
                                                                        K);
        return cuda_fail(cudaGetLastError(), "nep_md_get_shc");
    }
    return NEP_OK;
}

int nep_shc_spectrum(const double* K, int n_lags, double dt_lag, int n_omega, const double* omega, double scale,
                     int window, double* out, void* stream)
{
    if (!K || !omega || !out || n_lags < 1 || n_omega < 1 || !(dt_lag > 0.0)) {
        set_error("nep_shc_spectrum: bad arguments");
        return NEP_ERR_ARG;
    }
    const int e = n_omega * 3;
    k_shc_spectrum<<<(e + 127) / 128, 128, 0, (cudaStream_t)stream>>>(n_lags, K, dt_lag, n_omega, omega, 1.0,
                                                                      scale, window ? 1 : 0, out);
    return cuda_fail(cudaGetLastError(), "nep_shc_spectrum");
}

int nep_shc_quantum(const double* omega, int n_omega, double x_per_omega, double* spec, void* stream)
{
    if (!omega || !spec || n_omega < 1 || !std::isfinite(x_per_omega)) {
        set_error("nep_shc_quantum: bad arguments");
        return NEP_ERR_ARG;
    }
    k_shc_quantum<<<(n_omega + 127) / 128, 128, 0, (cudaStream_t)stream>>>(n_omega, omega, x_per_omega, spec);
    return cuda_fail(cudaGetLastError(), "nep_shc_quantum");
}

int nep_hnemd_kappa(const double* J, int n, double scale, double* out, void* stream)
{
    if (!J || !out || n < 1) {
        set_error("nep_hnemd_kappa: bad arguments");
        return NEP_ERR_ARG;
    }
    k_hnemd_kappa<<<1, kKappaThreads, 0, (cudaStream_t)stream>>>(n, J, scale, out);
    return cuda_fail(cudaGetLastError(), "nep_hnemd_kappa");
}

int nep_hnemd_kappa_si(const double* J, int n, double temperature, double volume, double fe, double* out,
                       void* stream)
{
    if (!J || !out || n < 1 || !(temperature > 0.0) || !(volume > 0.0) || !(fe != 0.0) ||
        !std::isfinite(temperature * volume * fe)) {
        set_error("nep_hnemd_kappa_si: bad arguments (T > 0, V > 0, F_e != 0, all finite)");
        return NEP_ERR_ARG;
    }
    // <J> / (T V F_e) in eV / (A fs K) = kEvPerAFsK_WPerMK W / (m K)
    const double scale = kEvPerAFsK_WPerMK / (temperature * volume * fe);
    k_hnemd_kappa<<<1, kKappaThreads, 0, (cudaStream_t)stream>>>(n, J, scale, out);
    return cuda_fail(cudaGetLastError(), "nep_hnemd_kappa_si");
}

int nep_kappa_spectrum(const double* K, int n_lags, double dt_lag_fs, const double* nu_thz, int n_nu,
                       double temperature, double volume, double fe, int window, int quantum, double* out,
                       void* stream)
{
    if (!K || !nu_thz || !out || n_lags < 1 || n_nu < 1 || !(dt_lag_fs > 0.0) || !(temperature > 0.0) ||
        !(volume > 0.0) || !(fe != 0.0) || !std::isfinite(temperature * volume * fe * dt_lag_fs)) {
        set_error("nep_kappa_spectrum: bad arguments (lags, frequencies >= 1; dt, T, V > 0; F_e != 0)");
        return NEP_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // omega = 2 pi nu, in rad/fs for nu in THz; kappa per THz of nu: the
    // W / (m K) of <J>/(T V F_e) times 1e-3 (the fs of dt over the ps of 1/nu)
    const double omega_per_nu = 2.0 * kPi * 1e-3;
    const double scale = 2.0 / (temperature * volume * fe) * kEvPerAFsK_WPerMK * 1e-3;
    const int e = n_nu * 3;
    k_shc_spectrum<<<(e + 127) / 128, 128, 0, st>>>(n_lags, K, dt_lag_fs, n_nu, nu_thz, omega_per_nu, scale,
                                                    window ? 1 : 0, out);
    // x = hbar omega / (k_B T) = (hbar / (k_B T)) (2 pi 1e-3) nu
    if (quantum)
        k_shc_quantum<<<(n_nu + 127) / 128, 128, 0, st>>>(
            n_nu, nu_thz, kHbarEvFs / (kBoltzmannEv * temperature) * omega_per_nu, out);
    return cuda_fail(cudaGetLastError(), "nep_kappa_spectrum");
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
    fa.nr = m->hp.n_max_R + 1;
    fa.na = m->hp.n_max_A + 1;
    fa.typed = md_zatom(md) != nullptr;
    if (m->zatom && !fa.typed) {
        set_error("nep_md_step: species were set for %d atoms, not %d", m->zatom_n, n);
        return NEP_ERR_ARG;
    }
    const double rmax = m->hp.rc_R > m->hp.rc_A ? m->hp.rc_R : m->hp.rc_A;
    const double conv = kAmuA2Fs2InEv;
    int rc;
    if (md->tau > 0.0 && n < 2) {
        set_error("nep_md_step: the thermostat needs at least two atoms");
        return NEP_ERR_ARG;
    }

    // site energies and partial forces: the optimised pass, or the plain FP32
    // comparator (literal Eq. 13, unfused) when selected
    Workspace& wsp = md->ws;
    auto site_pass = [&](cudaStream_t q, int& b1) {
        if (md->plain)
            return launch_plain_site(fa, nl, n, wsp.plain, wsp.plain + (size_t)kNdes * n, nullptr, part_e, m->d_err, q,
                                     b1);
        return launch_site_partial_forces(fa, nl, n, nullptr, part_e, m->d_err, q, b1);
    };
    if (md->need_init) {
        // forces of the starting configuration (list built unconditionally)
        if ((rc = build_neighbor_list(nl, md->box, n, pos, md_zatom(md), true, md->x_ref, md->r_list, m->d_err, nullptr, st)))
            return rc;
        int b1 = 0, b2 = 0, c2 = 0;
        if ((rc = site_pass(st, b1))) return rc;
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
    const double dof_kb = (3.0 * n - 3.0) * kBoltzmannEv;

    // one step in three parts: kick-drift and the rebuild decision, the list
    // rebuild, then forces, second half kick and the step's sums
    auto head = [&](cudaStream_t q, bool use_cond, cudaGraphConditionalHandle cond) {
        Profiler::Slot* pk = m->prof.begin(NEP_PROFILE_STEP, q);
        k_kick_drift<<<blocks_for(n, 256), 256, 0, q>>>(n, pos, vel, md->ws.force, hdtm, dt, nl.xh, nl.xl, md->x_ref,
                                                        md->ctl, thresh * thresh, md->rebuilds, cond,
                                                        use_cond ? 1 : 0);
        m->prof.end(pk, q);
    };
    auto rebuild = [&](cudaStream_t q, const unsigned* g) {
        Profiler::Slot* pk = m->prof.begin(NEP_PROFILE_NEIGHBOR, q);
        const int r = build_neighbor_list(nl, md->box, n, pos, md_zatom(md), true, md->x_ref, md->r_list, m->d_err, g, q);
        m->prof.end(pk, q);
        return r;
    };
    auto tail = [&](cudaStream_t q) {
        int b1 = 0, b2 = 0, c2 = 0, r;
        // spectral heat current: this step's W_i goes to the ring when sampled
        const bool sample = md->shc_lags > 0 && md->shc_step % md->shc_every == 0;
        const int slot = sample ? (int)(md->shc_samples % md->shc_lags) : 0;
        float* w_out = sample ? md->shc_ring + (size_t)slot * 9 * n : (drive ? md->w_atom : nullptr);
        Profiler::Slot* ps = m->prof.begin(NEP_PROFILE_SITE, q);
        if ((r = site_pass(q, b1))) return r;
        m->prof.end(ps, q);
        AssembleArgs aa{};
        aa.rc_max = (float)rmax;
        aa.box = md->box;
        aa.vel = drive ? nullptr : vel;  // with HNEMD the kick waits for the total virial
        aa.half_dt_over_m = hdtm;
        aa.ke_factor = kef;
        aa.heat = heat != nullptr;
        ps = m->prof.begin(NEP_PROFILE_ASSEMBLE, q);
        if ((r = launch_assemble(aa, nl, n, md->ws.force, w_out, part_a, m->d_err, q, b2, c2))) return r;
        m->prof.end(ps, q);
        Profiler::Slot* pk = m->prof.begin(NEP_PROFILE_STEP, q);
        if (drive) {
            // the kick needs the total virial first
            if ((r = launch_reduce(part_a, b2, c2, md->red + 1, q))) return r;
            k_hnemd_kick<<<nbk, 256, 0, q>>>(n, md->ws.force, w_out, vel, md->fe[0], md->fe[1], md->fe[2],
                                             md->red + 1, 1.0 / n, hdtm, kef, part_h, m->d_err);
            k_md_finish<<<5, kFinishThreads, 0, q>>>(part_e, b1, part_h, nbk, 4, 10, md->red, thermo, heat, md->ctl,
                                                     md->t0, md->tau, dt, dof_kb);
        } else {
            k_md_finish<<<1 + c2, kFinishThreads, 0, q>>>(part_e, b1, part_a, b2, c2, 1, md->red, thermo, heat,
                                                          md->ctl, md->t0, md->tau, dt, dof_kb);
        }
        if (sample) {  // v is that of J: after the second half kick, before the thermostat
            const int avail = (int)(md->shc_samples + 1 < md->shc_lags ? md->shc_samples + 1 : md->shc_lags);
            const int chunks = (n + kShcChunk - 1) / kShcChunk;
            k_shc_corr<<<dim3((avail + kShcLagsPerBlock - 1) / kShcLagsPerBlock, chunks), 32 * kShcLagsPerBlock, 0,
                         q>>>(n, md->shc_lags, avail, slot, md->shc_ring, vel, md->shc_part);
            k_shc_reduce<<<(avail * 3 + 127) / 128, 128, 0, q>>>(md->shc_lags, avail, chunks, md->shc_part,
                                                                  md->shc_sum);
            ++md->shc_samples;
        }
        if (md->shc_lags > 0) ++md->shc_step;
        if (md->tau > 0.0 && n > 1) k_scale_v<<<nbk, 256, 0, q>>>(n, vel, md->red);
        m->prof.end(pk, q);
        return cuda_fail(cudaGetLastError(), "md step kernels");
    };

    // Without phase timing and without the per-step host logic of the
    // spectral heat current, a step runs from a CUDA graph captured once: the
    // list rebuild is the body of a conditional node that the last block of
    // k_kick_drift switches,
    // so a step without a rebuild launches none of the list kernels.
    if (!m->prof.on && md->shc_lags == 0) {
        nep_md::GraphKey key{pos, vel, thermo, heat, dt, md->t0, md->tau, {md->fe[0], md->fe[1], md->fe[2]}, drive,
                             md_zatom(md), md->plain};
        if (!md->gexec || !(key == md->gkey)) {
            if (md->gexec) cudaGraphExecDestroy(md->gexec);
            md->gexec = nullptr;
            if (!md->gcap && (rc = cuda_fail(cudaStreamCreateWithFlags(&md->gcap, cudaStreamNonBlocking), "stream")))
                return rc;
            if (!md->gcap2 && (rc = cuda_fail(cudaStreamCreateWithFlags(&md->gcap2, cudaStreamNonBlocking), "stream")))
                return rc;
            cudaGraph_t g = nullptr;
            cudaGraphConditionalHandle cond;
            rc = cuda_fail(cudaGraphCreate(&g, 0), "graph create");
            if (!rc) rc = cuda_fail(cudaGraphConditionalHandleCreate(&cond, g, 0, cudaGraphCondAssignDefault), "handle");
            if (!rc) rc = cuda_fail(cudaStreamBeginCaptureToGraph(md->gcap, g, nullptr, nullptr, 0,
                                                                  cudaStreamCaptureModeRelaxed), "begin capture");
            if (rc) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            head(md->gcap, true, cond);
            cudaStreamCaptureStatus cs;
            const cudaGraphNode_t* deps = nullptr;
            size_t nd = 0;
            rc = cuda_fail(cudaStreamGetCaptureInfo(md->gcap, &cs, nullptr, nullptr, &deps, nullptr, &nd), "capture info");
            cudaGraphNodeParams cp = {};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = cond;
            cp.conditional.type = cudaGraphCondTypeIf;
            cp.conditional.size = 1;
            cudaGraphNode_t cnode = nullptr;
            if (!rc) rc = cuda_fail(cudaGraphAddNode(&cnode, g, deps, nullptr, nd, &cp), "conditional node");
            if (!rc)
                rc = cuda_fail(cudaStreamUpdateCaptureDependencies(md->gcap, &cnode, nullptr, 1,
                                                                   cudaStreamSetCaptureDependencies),
                               "capture dependencies");
            if (!rc) {
                cudaGraph_t body = cp.conditional.phGraph_out[0];
                rc = cuda_fail(cudaStreamBeginCaptureToGraph(md->gcap2, body, nullptr, nullptr, 0,
                                                             cudaStreamCaptureModeRelaxed), "begin body capture");
                if (!rc) {
                    rc = rebuild(md->gcap2, nullptr);
                    cudaGraph_t b2 = nullptr;
                    const cudaError_t e = cudaStreamEndCapture(md->gcap2, &b2);
                    if (!rc && e != cudaSuccess) rc = cuda_fail(e, "end body capture");
                }
            }
            if (!rc) rc = tail(md->gcap);
            cudaGraph_t g2 = nullptr;
            const cudaError_t e = cudaStreamEndCapture(md->gcap, &g2);
            if (!rc && e != cudaSuccess) rc = cuda_fail(e, "end capture");
            if (!rc) rc = cuda_fail(cudaGraphInstantiate(&md->gexec, g, 0), "instantiate step graph");
            cudaGraphDestroy(g);
            if (rc) {
                md->gexec = nullptr;
                return rc;
            }
            md->gkey = key;
        }
        for (int s = 0; s < n_steps; ++s)
            if ((rc = cuda_fail(cudaGraphLaunch(md->gexec, st), "launch step graph"))) return rc;
        return NEP_OK;
    }

    const unsigned* gate = md->ctl + kCtlGate;
    for (int s = 0; s < n_steps; ++s) {
        head(st, false, cudaGraphConditionalHandle{});
        if ((rc = rebuild(st, gate))) return rc;
        if ((rc = tail(st))) return rc;
    }
    return NEP_OK;
}

}  // extern "C"
