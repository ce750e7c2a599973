// nep_force.cu -- the FP32 force path: site energies + partial forces, then
// force / per-atom virial assembly, and deterministic FP64 reductions.
//
// Pass A (k_site): one thread per atom runs the descriptor sums, the network
// and the partial forces dU_i/dr_ij of all its pairs (nep_site.cuh); the
// parameter vector sits in shared memory where every lane reads the same
// word (broadcast).  Partial forces go to pf[k][i] as float4 records
// (coalesced per slot).
// Pass B (k_assemble): one thread per atom gathers its own p_ij and the
// neighbours' p_ji through the reverse-pair index: F_i = sum_j (p_ij - p_ji)
// and W_i = sum_j r_ij (x) p_ji (Eqs. 4-6).  In MD mode the same pass applies
// the second velocity-Verlet half kick and accumulates E_kin and the heat
// current J = sum_i W_i . v_i (Eq. 7) without storing W.
// Totals are summed per block in FP64 and then by one block in a fixed order,
// so every result is bitwise reproducible run to run.
#include <cstdio>

#include "nep_site.cuh"

namespace nep {

namespace {

constexpr int kSiteThreads = kSiteAtomsPerBlock;  // one thread per atom
constexpr int kAsmThreads = 128;
constexpr int kStageSlots = 96;  // slots per atom staged in shared memory
static_assert(kStageSlots <= 256, "original slot numbers are stored in one byte");

// Copy the block's neighbour slots (slot-major: slot k of the block's atoms is
// one contiguous run) into shared memory with 4-byte asynchronous copies, all
// in flight at once; slots past an atom's count are not read.
__device__ __forceinline__ void stage_slots(const int* __restrict__ nbr, int n, int i, bool active, int cnt,
                                            int* s_nbr)
{
    if (active)
        for (int k = 0; k < cnt; ++k) {
            int* dst = s_nbr + k * kSiteThreads + threadIdx.x;
            const int* src = nbr + (size_t)k * n + i;
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                         "l"(src)
                         : "memory");
        }
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_all;" ::: "memory");
}

// Compacts a thread's staged slot column (cnt entries, s_col[k * kSiteThreads])
// in place to the slots within rc2max, in their order, and records each kept
// entry's original slot in o_col; returns the number kept.  The test is the
// one the site passes apply (the same pair vector and distance square), so
// the passes see exactly the slots they would have used; slots beyond the
// cutoff (about 40 % of a Verlet list with a 1 A skin) then cost no loop
// iteration there.  Four slots are gathered at a time.  Bit k of mb is set
// for each kept slot k.
__device__ __forceinline__ int compact_slots(int i, int cnt, int* s_col, unsigned char* o_col,
                                             const float* __restrict__ xh, const float* __restrict__ xl, int n,
                                             const Box& box, float rc2max, unsigned (&mb)[3])
{
    mb[0] = mb[1] = mb[2] = 0u;
    float hi[3], li[3];
    load_pos(xh, xl, n, i, hi, li);
    int kept = 0;
    for (int k0 = 0; k0 < cnt; k0 += 4) {
        int v[4];
        float4 a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = (k0 + u < cnt) ? s_col[(k0 + u) * kSiteThreads] : 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = v[u] & 0xFFFFFF;  // 0 past the end: a valid atom
            a[u] = NEP_LDG(reinterpret_cast<const float4*>(xh) + j);
            b[u] = NEP_LDG(reinterpret_cast<const float4*>(xl) + j);
        }
        // every read of this group precedes the writes, and kept <= k0 + u
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (k0 + u < cnt) {
                const float hj[3] = {a[u].x, a[u].y, a[u].z}, lj[3] = {b[u].x, b[u].y, b[u].z};
                float rx, ry, rz;
                pair_vector(i, v[u] & 0xFFFFFF, v[u] >> 24, hi, li, hj, lj, box, rx, ry, rz);
                const float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                if (d2 < rc2max) {
                    s_col[kept * kSiteThreads] = v[u];
                    o_col[kept * kSiteThreads] = (unsigned char)(k0 + u);
                    ++kept;
                    const int k = k0 + u;
                    mb[k >> 5] |= 1u << (k & 31);
                }
            }
        }
    }
    return kept;
}

// STAGED: the neighbour capacity fits the shared-memory staging (m_cap <= kStageSlots).
// D: descriptor sizes of the model (DescSi: 32 descriptors, DescPbTe: 41).
template <bool STAGED, class D>
__global__ void __launch_bounds__(kSiteThreads) k_site(int n, int m_cap, const int* __restrict__ count,
                                                       const int* __restrict__ nbr, const float* __restrict__ xh,
                                                       const float* __restrict__ xl, Box box,
                                                       const float* __restrict__ z, int n_par, SiteParams P,
                                                       float* __restrict__ pf, double* __restrict__ e_atom,
                                                       double* __restrict__ e_partials, unsigned* err,
                                                       unsigned* __restrict__ mask)
{
    extern __shared__ float s_w[];
    for (int t = threadIdx.x; t < n_par; t += blockDim.x) s_w[t] = z[t];
    P.w = s_w;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double e[1] = {0.0};
    // every lane runs the site function (the warp walks neighbour ranks in
    // step); lanes past the last atom see no neighbours and store nothing
    const bool active = i < n;
    int cnt = active ? min(count[i], m_cap) : 0;
    int* s_nbr = reinterpret_cast<int*>(s_w + ((n_par + 31) / 32) * 32);
    unsigned char* s_orig = reinterpret_cast<unsigned char*>(s_nbr + kStageSlots * kSiteThreads);
    if (STAGED) {
        stage_slots(nbr, n, i, active, cnt, s_nbr);
        if (active) {
            unsigned mb[3];
            cnt = compact_slots(i, cnt, s_nbr + threadIdx.x, s_orig + threadIdx.x, xh, xl, n, box,
                                fmaxf(P.rcR2, P.rcA2), mb);
            if (mask) {
                mask[i] = mb[0];
                mask[(size_t)n + i] = mb[1];
                mask[(size_t)2 * n + i] = mb[2];
            }
        }
    }
    __syncthreads();
    const SlotTable T = STAGED ? SlotTable{s_nbr, kSiteThreads, (int)threadIdx.x, s_orig}
                               : SlotTable{nbr, n, i};
    float uh, ul;
    const PfOut out{pf + 4 * (size_t)(active ? i : 0), (size_t)4 * n, 1};
    site_partial_forces<D>(active ? i : 0, active, n, cnt, T, xh, xl, box, P, out, uh, ul);
    if (active) {
        e[0] = (double)uh + (double)ul;
        if (e_atom) e_atom[i] = e[0];
        if (!isfinite(uh)) atomicOr(err, kErrNonFinite);
    }
    block_sum_store<1>(e, e_partials + blockIdx.x);
}

// Totals per block: [0..8] virial, and in MD mode [9] E_kin, [10..12] J.
template <bool MD>
__global__ void __launch_bounds__(kAsmThreads) k_assemble(int n, int m_cap, float rc2max, const int* __restrict__ count,
                                                          const int* __restrict__ nbr, const int* __restrict__ rev,
                                                          const float* __restrict__ xh, const float* __restrict__ xl,
                                                          Box box, const float* __restrict__ pf,
                                                          float* __restrict__ force, float* __restrict__ virial_atom,
                                                          double* __restrict__ partials, unsigned* err,
                                                          double* __restrict__ vel, double hdtm, double kef,
                                                          const unsigned* __restrict__ mask)
{
    constexpr int K = MD ? 13 : 9;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    if (i < n) {
        // the list is read straight from global memory: staging it in shared
        // memory (as the site pass does) cost this pass occupancy and time
        const SlotTable T{nbr, n, i};
        float F[3], W[9];
        assemble_atom(i, n, m_cap, rc2max, count, T, rev, xh, xl, box, pf, F, W, mask);
        if (!(isfinite(F[0]) && isfinite(F[1]) && isfinite(F[2]))) atomicOr(err, kErrNonFinite);
        if (force) {
            force[i] = F[0];
            force[(size_t)n + i] = F[1];
            force[(size_t)2 * n + i] = F[2];
        }
        if (virial_atom)
#pragma unroll
            for (int c = 0; c < 9; ++c) virial_atom[(size_t)c * n + i] = W[c];
#pragma unroll
        for (int c = 0; c < 9; ++c) acc[c] = (double)W[c];
        if constexpr (MD) {
            double v[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                v[c] = vel[(size_t)c * n + i] + hdtm * (double)F[c];
                vel[(size_t)c * n + i] = v[c];
            }
            acc[9] = kef * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            // J^a = sum_b W^{ab} v^b, FP32 products accumulated in FP64
#pragma unroll
            for (int a = 0; a < 3; ++a)
                acc[10 + a] = (double)(W[3 * a] * (float)v[0]) + (double)(W[3 * a + 1] * (float)v[1]) +
                              (double)(W[3 * a + 2] * (float)v[2]);
        }
    }
    block_sum_store<K>(acc, partials + (size_t)blockIdx.x * K);
}

// out[k] = sum_b partials[b * ncomp + k]: one warp per component, each lane
// summing a fixed stride of blocks, then a fixed shuffle tree (deterministic).
__global__ void k_reduce(const double* __restrict__ partials, int nblocks, int ncomp, double* __restrict__ out)
{
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (k >= ncomp) return;
    double s = 0.0;
    // unrolled so that eight loads are in flight ahead of the (ordered) adds
#pragma unroll 8
    for (int b = lane; b < nblocks; b += 32) s += partials[(size_t)b * ncomp + k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[k] = s;
}

inline int blocks_for(int n, int t) { return (n + t - 1) / t; }

template <class D>
int launch_site(const ForceArgs& a, NeighborList& nl, int n, double* e_atom, double* e_partials, unsigned* d_err,
                cudaStream_t st, int& nblocks)
{
    SiteParams P;
    P.w = nullptr;
    P.n_neu = a.n_neu;
    P.rcR = a.rcR;
    P.rcA = a.rcA;
    P.rcR2 = a.rcR * a.rcR;
    P.rcA2 = a.rcA * a.rcA;
    P.inv_rcR = 1.f / a.rcR;
    P.inv_rcA = 1.f / a.rcA;
    P.typed = a.typed;
    const int n_par = (D::Ndes + 2) * a.n_neu + 1;
    nblocks = blocks_for(n, kSiteThreads);
    // weights, the staged slots and their original slot numbers (one byte each)
    const size_t smem = (((size_t)n_par + 31) / 32 * 32 + (size_t)kStageSlots * kSiteThreads) * sizeof(float) +
                        (size_t)kStageSlots * kSiteThreads;
    const bool staged = a.box.nc[0] >= 0 && nl.m_cap <= kStageSlots;
    if (staged) {
        int rc = cuda_fail(cudaFuncSetAttribute(k_site<true, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                           "site kernel shared memory");
        if (rc) return rc;
    }
    auto kern = staged ? k_site<true, D> : k_site<false, D>;
    kern<<<nblocks, kSiteThreads, staged ? smem : (((size_t)n_par + 31) / 32 * 32) * sizeof(float), st>>>(
        n, nl.m_cap, nl.count, nl.nbr, nl.xh, nl.xl, a.box, a.z, n_par, P, nl.pf, e_atom, e_partials, d_err,
        staged ? nl.mask : nullptr);
    nl.mask_set = staged && nl.mask != nullptr;
    return cuda_fail(cudaGetLastError(), "site kernel");
}

}  // namespace

int launch_site_partial_forces(const ForceArgs& a, NeighborList& nl, int n, double* e_atom, double* e_partials,
                               unsigned* d_err, cudaStream_t st, int& nblocks)
{
    if (a.nr == DescPbTe::NR && a.na == DescPbTe::NA)
        return launch_site<DescPbTe>(a, nl, n, e_atom, e_partials, d_err, st, nblocks);
    if (a.nr != DescSi::NR || a.na != DescSi::NA) {
        set_error("no site kernel for %d radial and %d angular orders", a.nr, a.na);
        return NEP_ERR_UNSUPPORTED;
    }
    return launch_site<DescSi>(a, nl, n, e_atom, e_partials, d_err, st, nblocks);
}

int launch_assemble(const AssembleArgs& a, NeighborList& nl, int n, float* force, float* virial_atom,
                    double* partials, unsigned* d_err, cudaStream_t st, int& nblocks, int& ncomp)
{
    nblocks = blocks_for(n, kAsmThreads);
    const float rc2 = a.rc_max * a.rc_max;
    const bool md = a.vel != nullptr;
    ncomp = md ? 13 : 9;
    auto kern = md ? k_assemble<true> : k_assemble<false>;
    kern<<<nblocks, kAsmThreads, 0, st>>>(n, nl.m_cap, rc2, nl.count, nl.nbr, nl.rev, nl.xh, nl.xl, a.box, nl.pf,
                                          force, virial_atom, partials, d_err, md ? a.vel : nullptr,
                                          md ? a.half_dt_over_m : 0.0, md ? a.ke_factor : 0.0,
                                          nl.mask_set ? nl.mask : nullptr);
    return cuda_fail(cudaGetLastError(), "assemble kernel");
}

int launch_reduce(const double* partials, int nblocks, int ncomp, double* out, cudaStream_t st)
{
    k_reduce<<<1, 32 * ncomp, 0, st>>>(partials, nblocks, ncomp, out);
    return cuda_fail(cudaGetLastError(), "reduce kernel");
}

}  // namespace nep
