// nep_api.cu -- the C ABI of include/nep.h: argument checks, handles,
// device scratch, and the single-configuration entry points.
#include <cmath>
#include <vector>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "nep_internal.cuh"

namespace nep {

namespace {
thread_local char g_err[512] = "";

__global__ void k_finish_efv(const double* __restrict__ red, double* e_total, double* virial_total)
{
    if (threadIdx.x == 0 && e_total) *e_total = red[0];
    if (threadIdx.x < 9 && virial_total) virial_total[threadIdx.x] = red[1 + threadIdx.x];
}

// J^a = sum_i sum_b W_i^{ab} v_i^b per block, FP32 products, FP64 sums.
__global__ void k_heat(int n, const float* __restrict__ W, const double* __restrict__ v, double* __restrict__ part)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double J[3] = {0.0, 0.0, 0.0};
    if (i < n) {
        float vv[3];
        for (int b = 0; b < 3; ++b) vv[b] = (float)v[(size_t)b * n + i];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) J[a] += (double)(W[(size_t)(3 * a + b) * n + i] * vv[b]);
    }
    block_sum_store<3>(J, part + (size_t)blockIdx.x * 3);
}

template <class T>
int dev_alloc(T** p, size_t count, const char* what)
{
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        set_error("cudaMalloc of %zu bytes for %s failed: %s", count * sizeof(T), what, cudaGetErrorString(e));
        return NEP_ERR_OOM;
    }
    return NEP_OK;
}

template <class T>
void dev_free(T*& p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

int check_hyper(const nep_hyper* hp)
{
    if (!hp) {
        set_error("hyperparameters are NULL");
        return NEP_ERR_ARG;
    }
    if (!(hp->rc_R > 0.0) || !(hp->rc_A > 0.0) || !(hp->skin >= 0.0) || hp->max_neighbors < 1 ||
        hp->max_neighbors > 384 || hp->n_neu < 1) {
        set_error("invalid hyperparameters (cutoffs > 0, skin >= 0, 1 <= max_neighbors <= 384, n_neu >= 1)");
        return NEP_ERR_ARG;
    }
    if (!(sizes_default(*hp) || sizes_split(*hp)) || hp->l_max != kLmax || hp->n_neu > kMaxNeu) {
        set_error("this build has kernels for (n_max_R, n_max_A) = (%d, %d) or (12, 6), l_max=%d, n_neu<=%d",
                  kNR - 1, kNA - 1, kLmax, kMaxNeu);
        return NEP_ERR_UNSUPPORTED;
    }
    return NEP_OK;
}

}  // namespace

void set_error(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int cuda_fail(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return NEP_OK;
    set_error("%s: %s", what, cudaGetErrorString(e));
    return NEP_ERR_CUDA;
}

int status_from_bits(unsigned bits)
{
    if (bits & kErrOverflow) {
        set_error("an atom had more neighbours than max_neighbors");
        return NEP_ERR_NEIGHBOR_OVERFLOW;
    }
    if (bits & kErrReverse) {
        set_error("neighbour list not symmetric (reverse pair missing)");
        return NEP_ERR_NEIGHBOR_OVERFLOW;
    }
    if (bits & kErrNonFinite) {
        set_error("non-finite position, site energy or force (or a force term beyond the fixed-point range)");
        return NEP_ERR_NONFINITE;
    }
    if (bits & kErrTimeout) {
        set_error("a bounded device wait timed out");
        return NEP_ERR_TIMEOUT;
    }
    return NEP_OK;
}

int setup_box(const double* box9, double r_list, Box& b)
{
    if (!box9) {
        set_error("box is NULL");
        return NEP_ERR_ARG;
    }
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            if (r != c && box9[3 * r + c] != 0.0) {
                set_error("only orthorhombic boxes are supported (off-diagonal box entries must be 0)");
                return NEP_ERR_BOX;
            }
    bool cells = true;
    long long nc[3] = {0, 0, 0};
    for (int d = 0; d < 3; ++d) {
        const double L = box9[4 * d];
        if (!(L > 0.0) || !std::isfinite(L)) {
            set_error("box edge %d is not positive", d);
            return NEP_ERR_BOX;
        }
        if (L < 0.5 * r_list) {
            set_error("box edge %d (%.4g A) is shorter than half the neighbour radius (%.4g A)", d, L, r_list);
            return NEP_ERR_BOX;
        }
        b.L[d] = L;
        split_hilo(L, b.Lh[d], b.Ll[d]);
        // cells per direction, counted in 64 bits (L / r_list can exceed an int)
        const double f = std::floor(L / r_list);
        nc[d] = f > (double)kMaxCells ? (long long)kMaxCells : (long long)f;
        if (nc[d] < 3) cells = false;
        b.img[d] = (int)std::ceil(r_list / L);
        if (b.img[d] > 2) b.img[d] = 2;
    }
    // coarsen the grid until it has at most kMaxCells cells: halving the
    // longest direction keeps every cell edge >= r_list, and a direction over
    // the cube root of the cap (161) never drops below 3 cells
    while (cells && nc[0] * nc[1] * nc[2] > (long long)kMaxCells) {
        const int d = (nc[0] >= nc[1] && nc[0] >= nc[2]) ? 0 : (nc[1] >= nc[2] ? 1 : 2);
        nc[d] = (nc[d] + 1) / 2;
    }
    for (int d = 0; d < 3; ++d) b.nc[d] = cells ? (int)nc[d] : 0;
    for (int d = 0; d < 3; ++d) b.cpl[d] = b.nc[d] / b.L[d];
    return NEP_OK;
}

// Grows the scratch to hold n atoms with m_cap slots, ncell cells and the
// per-block partial sums of nblocks blocks (16 doubles per block).
int ensure_workspace(Workspace& ws, int n, int m_cap, int ncell, int nblocks_partials)
{
    NeighborList& nl = ws.nl;
    int rc = NEP_OK;
    if (n > nl.n_cap || m_cap != nl.m_cap) {
        dev_free(nl.count);
        dev_free(nl.nbr);
        dev_free(nl.rev);
        dev_free(nl.vala);
        dev_free(nl.pf);
        dev_free(nl.xh);
        dev_free(nl.xl);
        dev_free(nl.atom_cell);
        dev_free(nl.cell_atoms);
        dev_free(nl.mask);
        dev_free(ws.force);
        nl.n_cap = nl.m_cap = 0;
        ws.force_cap = 0;
        const size_t N = (size_t)n, M = (size_t)m_cap;
        if ((rc = dev_alloc(&nl.count, N, "neighbour counts")) || (rc = dev_alloc(&nl.nbr, N * M, "neighbour list")) ||
            (rc = dev_alloc(&nl.rev, N * M, "reverse pair index")) ||
            (rc = dev_alloc(&nl.vala, N * M, "neighbour list copy")) ||
            (rc = dev_alloc(&nl.pf, N * M * 4, "partial forces")) || (rc = dev_alloc(&nl.xh, N * 4, "positions")) ||
            (rc = dev_alloc(&nl.xl, N * 4, "positions")) || (rc = dev_alloc(&nl.atom_cell, N, "cell index")) ||
            (rc = dev_alloc(&nl.cell_atoms, N, "cell atoms")) || (rc = dev_alloc(&nl.mask, N * 3, "slot masks")) ||
            (rc = dev_alloc(&ws.force, N * 3, "forces")))
            return rc;
        nl.n_cap = n;
        nl.m_cap = m_cap;
        ws.force_cap = n;
    }
    if (ncell + 1 > nl.ncell_cap) {
        dev_free(nl.cell_count);
        dev_free(nl.cell_start);
        dev_free(nl.cell_fill);
        nl.ncell_cap = 0;
        const size_t C = (size_t)ncell + 1;
        if ((rc = dev_alloc(&nl.cell_count, C, "cell counts")) || (rc = dev_alloc(&nl.cell_start, C, "cell offsets")) ||
            (rc = dev_alloc(&nl.cell_fill, C, "cell fill")))
            return rc;
        // the builder keeps both arrays zero between builds
        if ((rc = cuda_fail(cudaMemset(nl.cell_count, 0, C * sizeof(int)), "cudaMemset")) ||
            (rc = cuda_fail(cudaMemset(nl.cell_fill, 0, C * sizeof(int)), "cudaMemset")))
            return rc;
        nl.ncell_cap = (int)C;
    }
    const int need_partials = 16 * (nblocks_partials + 8);
    if (need_partials > ws.partial_cap) {
        dev_free(ws.partials);
        ws.partial_cap = 0;
        if ((rc = dev_alloc(&ws.partials, (size_t)need_partials, "partial sums"))) return rc;
        ws.partial_cap = need_partials;
    }
    return NEP_OK;
}

void free_workspace(Workspace& ws)
{
    NeighborList& nl = ws.nl;
    dev_free(nl.count);
    dev_free(nl.nbr);
    dev_free(nl.rev);
    dev_free(nl.vala);
    dev_free(nl.pf);
    dev_free(nl.xh);
    dev_free(nl.xl);
    dev_free(nl.atom_cell);
    dev_free(nl.cell_count);
    dev_free(nl.cell_start);
    dev_free(nl.cell_fill);
    dev_free(nl.cell_atoms);
    dev_free(nl.mask);
    dev_free(ws.partials);
    dev_free(ws.force);
    dev_free(ws.plain);
    nl = NeighborList();
    ws.partial_cap = ws.force_cap = ws.plain_cap = 0;
}

Profiler::Slot* Profiler::begin(int kind, cudaStream_t st)
{
    if (!on) return nullptr;
    if (used == cap) {
        const int ncap = cap ? 2 * cap : 256;
        Slot* ns = new (std::nothrow) Slot[ncap];
        if (!ns) return nullptr;
        for (int k = 0; k < cap; ++k) ns[k] = slots[k];
        for (int k = cap; k < ncap; ++k) {
            if (cudaEventCreate(&ns[k].a) != cudaSuccess || cudaEventCreate(&ns[k].b) != cudaSuccess) {
                cudaGetLastError();
                delete[] ns;
                return nullptr;
            }
        }
        delete[] slots;
        slots = ns;
        cap = ncap;
    }
    Slot* s = &slots[used++];
    s->kind = kind;
    cudaEventRecord(s->a, st);
    return s;
}

void Profiler::end(Slot* s, cudaStream_t st)
{
    if (s) cudaEventRecord(s->b, st);
}

int Profiler::read(double* ms, long long* cnt)
{
    for (int k = 0; k < NEP_PROFILE_KINDS; ++k) {
        ms[k] = 0.0;
        cnt[k] = 0;
    }
    for (int k = 0; k < used; ++k) {
        int rc = cuda_fail(cudaEventSynchronize(slots[k].b), "event synchronise");
        if (rc) return rc;
        float t = 0.f;
        if ((rc = cuda_fail(cudaEventElapsedTime(&t, slots[k].a, slots[k].b), "event elapsed time"))) return rc;
        ms[slots[k].kind] += t;
        cnt[slots[k].kind] += 1;
    }
    used = 0;
    return NEP_OK;
}

void Profiler::release()
{
    for (int k = 0; k < cap; ++k) {
        cudaEventDestroy(slots[k].a);
        cudaEventDestroy(slots[k].b);
    }
    delete[] slots;
    slots = nullptr;
    cap = used = 0;
}

}  // namespace nep

using namespace nep;

extern "C" {

const char* nep_last_error(void) { return g_err; }

int nep_create(const nep_hyper* hp, const float* z, int n_par, nep_model** out)
{
    g_err[0] = 0;
    if (!out || !z) {
        set_error("nep_create: NULL argument");
        return NEP_ERR_ARG;
    }
    *out = nullptr;
    int rc = check_hyper(hp);
    if (rc) return rc;
    const int n_des = (hp->n_max_R + 1) + (hp->n_max_A + 1) * hp->l_max;
    const int want = (n_des + 2) * hp->n_neu + 1;
    if (n_par != want) {
        set_error("nep_create: n_par = %d but (N_des + 2) N_neu + 1 = %d", n_par, want);
        return NEP_ERR_ARG;
    }
    nep_model* m = new (std::nothrow) nep_model();
    if (!m) {
        set_error("nep_create: host allocation failed");
        return NEP_ERR_OOM;
    }
    m->hp = *hp;
    m->n_des = n_des;
    m->n_par = n_par;
    if ((rc = dev_alloc(&m->d_z, (size_t)n_par, "parameters")) || (rc = dev_alloc(&m->d_err, 1, "error word")) ||
        (rc = dev_alloc(&m->d_red, 32, "reduction"))) {
        nep_destroy(m);
        return rc;
    }
    if ((rc = cuda_fail(cudaMemcpy(m->d_z, z, sizeof(float) * n_par, cudaMemcpyHostToDevice), "copy parameters")) ||
        (rc = cuda_fail(cudaMemset(m->d_err, 0, sizeof(unsigned)), "cudaMemset"))) {
        nep_destroy(m);
        return rc;
    }
    *out = m;
    return NEP_OK;
}

int nep_set_parameters(nep_model* m, const float* z, int n_par, void* stream)
{
    if (!m || !z || n_par != m->n_par) {
        set_error("nep_set_parameters: bad arguments");
        return NEP_ERR_ARG;
    }
    return cuda_fail(cudaMemcpyAsync(m->d_z, z, sizeof(float) * n_par, cudaMemcpyHostToDevice, (cudaStream_t)stream),
                     "copy parameters");
}

int nep_destroy(nep_model* m)
{
    if (!m) return NEP_OK;
    cudaDeviceSynchronize();
    m->prof.release();
    free_workspace(m->ws);
    dev_free(m->d_z);
    dev_free(m->d_err);
    dev_free(m->d_red);
    dev_free(m->zatom);
    delete m;
    return NEP_OK;
}

int nep_set_species(nep_model* m, int n, const double* z_atom)
{
    if (!m || n < 0 || n > kMaxAtoms || (n > 0 && !z_atom)) {
        set_error("nep_set_species: bad arguments");
        return NEP_ERR_ARG;
    }
    std::vector<float> zf((size_t)n);
    for (int i = 0; i < n; ++i) {
        if (!(z_atom[i] > 0.0) || !std::isfinite(z_atom[i])) {
            set_error("nep_set_species: the species number of atom %d is not positive", i);
            return NEP_ERR_ARG;
        }
        zf[(size_t)i] = (float)z_atom[i];
    }
    cudaDeviceSynchronize();
    dev_free(m->zatom);
    m->zatom_n = 0;
    if (n == 0) return NEP_OK;
    int rc = dev_alloc(&m->zatom, (size_t)n, "species numbers");
    if (rc) return rc;
    if ((rc = cuda_fail(cudaMemcpy(m->zatom, zf.data(), sizeof(float) * (size_t)n, cudaMemcpyHostToDevice),
                        "species upload"))) {
        dev_free(m->zatom);
        return rc;
    }
    m->zatom_n = n;
    return NEP_OK;
}

int nep_sync_status(nep_model* m, void* stream)
{
    if (!m) {
        set_error("nep_sync_status: NULL handle");
        return NEP_ERR_ARG;
    }
    int rc = cuda_fail(cudaStreamSynchronize((cudaStream_t)stream), "stream synchronise");
    if (rc) return rc;
    unsigned bits = 0;
    if ((rc = cuda_fail(cudaMemcpy(&bits, m->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost), "read error word")))
        return rc;
    if (bits) cudaMemset(m->d_err, 0, sizeof(unsigned));
    return status_from_bits(bits);
}

}  // extern "C"

namespace {

int compute_efv(nep_model* m, int n, const double* box9, const double* pos, double* e_total, double* e_atom,
                float* force, float* virial_atom, double* virial_total, void* stream, bool plain)
{
    if (!m || !pos || n < 1 || n > kMaxAtoms) {
        set_error("nep_compute_efv: bad arguments (handle, positions, 1 <= n < 2^24)");
        return NEP_ERR_ARG;
    }
    if (m->zatom && n != m->zatom_n) {
        set_error("nep_compute_efv: species were set for %d atoms, not %d (nep_set_species)", m->zatom_n, n);
        return NEP_ERR_ARG;
    }
    if (plain && !sizes_default(m->hp)) {
        set_error("nep_compute_efv_plain: the plain comparator has kernels for the 32-descriptor model only");
        return NEP_ERR_UNSUPPORTED;
    }
    if (m->zatom && plain) {
        set_error("nep_compute_efv_plain: the plain comparator has one species only");
        return NEP_ERR_UNSUPPORTED;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const double rmax = m->hp.rc_R > m->hp.rc_A ? m->hp.rc_R : m->hp.rc_A;
    Box box;
    int rc = setup_box(box9, rmax, box);
    if (rc) return rc;
    const int ncell = box.nc[0] * box.nc[1] * box.nc[2];
    const int nblocks = site_blocks(n);
    if ((rc = ensure_workspace(m->ws, n, m->hp.max_neighbors, ncell, nblocks))) return rc;
    NeighborList& nl = m->ws.nl;
    Profiler::Slot* pn = m->prof.begin(NEP_PROFILE_NEIGHBOR, st);
    if ((rc = build_neighbor_list(nl, box, n, const_cast<double*>(pos), m->zatom, false, nullptr, (float)rmax,
                                  m->d_err, nullptr, st)))
        return rc;
    m->prof.end(pn, st);
    ForceArgs fa{m->d_z, m->hp.n_neu, (float)m->hp.rc_R, (float)m->hp.rc_A, box};
    fa.nr = m->hp.n_max_R + 1;
    fa.na = m->hp.n_max_A + 1;
    fa.typed = m->zatom != nullptr;
    // partial sums: energies in [0, nblocks), assembly totals after them
    double* part_e = m->ws.partials;
    double* part_v = m->ws.partials + ((nblocks + 7) / 8) * 8;
    int nb1 = 0;
    Profiler::Slot* ps = m->prof.begin(NEP_PROFILE_SITE, st);
    if (plain) {
        Workspace& ws = m->ws;
        if (ws.plain_cap < n) {
            if (ws.plain) cudaFree(ws.plain);
            ws.plain = nullptr;
            ws.plain_cap = 0;
            cudaError_t e = cudaMalloc((void**)&ws.plain, sizeof(float) * 2 * kNdes * (size_t)n);
            if (e != cudaSuccess) {
                cudaGetLastError();
                set_error("nep_compute_efv_plain: scratch allocation failed");
                return NEP_ERR_OOM;
            }
            ws.plain_cap = n;
        }
        if ((rc = launch_plain_site(fa, nl, n, ws.plain, ws.plain + (size_t)kNdes * n, e_atom, part_e, m->d_err, st,
                                    nb1)))
            return rc;
    } else if ((rc = launch_site_partial_forces(fa, nl, n, e_atom, part_e, m->d_err, st, nb1))) {
        return rc;
    }
    m->prof.end(ps, st);
    AssembleArgs aa{};
    aa.rc_max = (float)rmax;
    aa.box = box;
    aa.vel = nullptr;
    int nb2 = 0, nc2 = 0;
    ps = m->prof.begin(NEP_PROFILE_ASSEMBLE, st);
    if ((rc = launch_assemble(aa, nl, n, force, virial_atom, part_v, m->d_err, st, nb2, nc2))) return rc;
    m->prof.end(ps, st);
    if (e_total || virial_total) {
        if ((rc = launch_reduce(part_e, nb1, 1, m->d_red, st))) return rc;
        if ((rc = launch_reduce(part_v, nb2, nc2, m->d_red + 1, st))) return rc;
        k_finish_efv<<<1, 32, 0, st>>>(m->d_red, e_total, virial_total);
        if ((rc = cuda_fail(cudaGetLastError(), "finish kernel"))) return rc;
    }
    return NEP_OK;
}

}  // namespace

extern "C" {

int nep_compute_efv(nep_model* m, int n, const double* box9, const double* pos, double* e_total, double* e_atom,
                    float* force, float* virial_atom, double* virial_total, void* stream)
{
    return compute_efv(m, n, box9, pos, e_total, e_atom, force, virial_atom, virial_total, stream, false);
}

int nep_compute_efv_plain(nep_model* m, int n, const double* box9, const double* pos, double* e_total,
                          double* e_atom, float* force, float* virial_atom, double* virial_total, void* stream)
{
    return compute_efv(m, n, box9, pos, e_total, e_atom, force, virial_atom, virial_total, stream, true);
}

int nep_profile_enable(nep_model* m, int on)
{
    if (!m) {
        set_error("nep_profile_enable: NULL handle");
        return NEP_ERR_ARG;
    }
    m->prof.on = on != 0;
    return NEP_OK;
}

int nep_profile_read(nep_model* m, double* ms, long long* launches)
{
    if (!m) {
        set_error("nep_profile_read: NULL handle");
        return NEP_ERR_ARG;
    }
    double t[NEP_PROFILE_KINDS];
    long long c[NEP_PROFILE_KINDS];
    int rc = m->prof.read(t, c);
    if (rc) return rc;
    for (int k = 0; k < NEP_PROFILE_KINDS; ++k) {
        if (ms) ms[k] = t[k];
        if (launches) launches[k] = c[k];
    }
    return NEP_OK;
}

int nep_status_from_bits(unsigned bits) { return status_from_bits(bits); }

int nep_cell_grid(const double* box9, double r_list, int* nc)
{
    if (!nc || !(r_list > 0.0) || !std::isfinite(r_list)) {
        set_error("nep_cell_grid: NULL output or a list radius that is not positive and finite");
        return NEP_ERR_ARG;
    }
    Box b;
    const int rc = setup_box(box9, r_list, b);
    if (rc) return rc;
    for (int d = 0; d < 3; ++d) nc[d] = b.nc[d];
    return NEP_OK;
}

int nep_get_neighbors(nep_model* m, int n, int* count, int* nbr, void* stream)
{
    if (!m || !count || !nbr || n < 1 || n > m->ws.nl.n_cap) {
        set_error("nep_get_neighbors: bad arguments (n must match the last nep_compute_efv call)");
        return NEP_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const NeighborList& nl = m->ws.nl;
    int rc = cuda_fail(cudaMemcpyAsync(count, nl.count, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, st),
                       "copy neighbour counts");
    if (rc) return rc;
    return cuda_fail(cudaMemcpyAsync(nbr, nl.nbr, sizeof(int) * (size_t)n * nl.m_cap, cudaMemcpyDeviceToDevice, st),
                     "copy neighbour list");
}

int nep_heat_current(nep_model* m, int n, const float* virial_atom, const double* vel, double* J, void* stream)
{
    if (!m || !virial_atom || !vel || !J || n < 1 || n > kMaxAtoms) {
        set_error("nep_heat_current: bad arguments");
        return NEP_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = (n + 255) / 256;
    int rc;
    if ((rc = ensure_workspace(m->ws, m->ws.nl.n_cap > 0 ? m->ws.nl.n_cap : 1,
                               m->ws.nl.m_cap > 0 ? m->ws.nl.m_cap : m->hp.max_neighbors, 0, nb)))
        return rc;
    k_heat<<<nb, 256, 0, st>>>(n, virial_atom, vel, m->ws.partials);
    if ((rc = cuda_fail(cudaGetLastError(), "heat-current kernel"))) return rc;
    return launch_reduce(m->ws.partials, nb, 3, J, st);
}

}  // extern "C"
