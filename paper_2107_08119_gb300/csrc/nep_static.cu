// nep_static.cu -- nep_compute_efv_static: the single-configuration force
// path for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need forces:
// code running while a memory pool is locked or exhausted by design, plugins
// whose host application owns every allocation, or hard real-time loops
// that forbid allocator calls.  This variant takes its scratch (neighbour
// list, reverse index, partial forces, FP32 positions, cells, partial sums)
// from one file-scope device array of fixed size instead of a handle's
// allocations, and needs no model handle: the caller passes the parameters,
// inputs and outputs, all in memory it already owns.
//
// Limits: at most NEP_STATIC_MAX_ATOMS atoms, NEP_STATIC_MAX_NEIGHBORS slots
// per atom and NEP_STATIC_MAX_CELLS cells (about 11.6 MB, resident on every
// GPU that loads the library until the process exits).  Every call shares
// the array, which keeps the previous call's contents; calls that overlap on
// the GPU (different streams, or host threads without ordering) race on it.
#include <cuda.h>

#include <mutex>

#include "nep_internal.cuh"

namespace nep {
namespace {

constexpr int kStaticAtoms = NEP_STATIC_MAX_ATOMS;
constexpr int kStaticSlots = NEP_STATIC_MAX_NEIGHBORS;
constexpr int kStaticCells = NEP_STATIC_MAX_CELLS;
constexpr int kStaticBlocks = (kStaticAtoms + kSiteAtomsPerBlock - 1) / kSiteAtomsPerBlock;

constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// byte offsets of every buffer inside the array
constexpr size_t kOffCount = 0;
constexpr size_t kOffNbr = kOffCount + align256(sizeof(int) * kStaticAtoms);
constexpr size_t kOffRev = kOffNbr + align256(sizeof(int) * kStaticAtoms * kStaticSlots);
constexpr size_t kOffVala = kOffRev + align256(sizeof(int) * kStaticAtoms * kStaticSlots);
constexpr size_t kOffPf = kOffVala + align256(sizeof(int) * kStaticAtoms * kStaticSlots);
constexpr size_t kOffXh = kOffPf + align256(sizeof(float) * kStaticAtoms * kStaticSlots * 4);
constexpr size_t kOffXl = kOffXh + align256(sizeof(float) * kStaticAtoms * 4);
constexpr size_t kOffAtomCell = kOffXl + align256(sizeof(float) * kStaticAtoms * 4);
constexpr size_t kOffCellAtoms = kOffAtomCell + align256(sizeof(int) * kStaticAtoms);
constexpr size_t kOffCellCount = kOffCellAtoms + align256(sizeof(int) * kStaticAtoms);
constexpr size_t kOffCellStart = kOffCellCount + align256(sizeof(int) * (kStaticCells + 1));
constexpr size_t kOffCellFill = kOffCellStart + align256(sizeof(int) * (kStaticCells + 1));
constexpr size_t kOffPartials = kOffCellFill + align256(sizeof(int) * (kStaticCells + 1));
constexpr size_t kOffRed = kOffPartials + align256(sizeof(double) * 16 * (kStaticBlocks + 8));
constexpr size_t kOffErr = kOffRed + align256(sizeof(double) * 32);
constexpr size_t kStaticBytes = kOffErr + align256(sizeof(unsigned));

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

// The array's device address belongs to a CUDA context (the module is loaded
// once per context).  It is cached per context, keyed by the driver's context
// id, which is unique for the life of the process: a new context -- after
// cudaDeviceReset, or a caller's own driver-API context -- gets a new id and
// a fresh lookup, never a stale address.  The two driver calls come through
// the runtime's entry-point query, so the library needs no libcuda link.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

constexpr int kCachedContexts = 16;
struct ScratchEntry {
    unsigned long long ctx_id;
    unsigned char* addr;
};
std::mutex g_setup_mutex;
ScratchEntry g_scratch_cache[kCachedContexts] = {};
int g_scratch_next = 0;
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
bool g_driver_queried = false;

// Id of the calling thread's current context, 0 if none is current or the
// driver calls are unavailable.  Caller holds g_setup_mutex.
unsigned long long current_context_id()
{
    if (!g_driver_queried) {
        g_driver_queried = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f);
        cudaGetLastError();
    }
    if (!g_ctx_get_current || !g_ctx_get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (g_ctx_get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the array in the current context.  In host code the
// array's name is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress, with the context (and its device) current.  The
// first call in a context does that lookup; later calls in it hit the cache.
int scratch_address(unsigned char** out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    unsigned long long id = current_context_id();
    if (id)
        for (int k = 0; k < kCachedContexts; ++k)
            if (g_scratch_cache[k].ctx_id == id) {
                *out = g_scratch_cache[k].addr;
                return NEP_OK;
            }
    void* p = nullptr;
    const int rc = cuda_fail(cudaGetSymbolAddress(&p, g_static_scratch), "cudaGetSymbolAddress of the static scratch");
    if (rc) return rc;
    // the lookup made the runtime's context current if none was
    if (!id) id = current_context_id();
    if (id) {
        g_scratch_cache[g_scratch_next] = ScratchEntry{id, static_cast<unsigned char*>(p)};
        g_scratch_next = (g_scratch_next + 1) % kCachedContexts;
    }
    *out = static_cast<unsigned char*>(p);
    return NEP_OK;
}

__global__ void k_static_finish(const double* __restrict__ red, double* e_total, double* virial_total,
                                const unsigned* __restrict__ err, unsigned* err_out)
{
    if (threadIdx.x == 0 && e_total) *e_total = red[0];
    if (threadIdx.x < 9 && virial_total) virial_total[threadIdx.x] = red[1 + threadIdx.x];
    if (threadIdx.x == 0 && err_out) *err_out = *err;
}

}  // namespace
}  // namespace nep

using namespace nep;

extern "C" int nep_compute_efv_static(const nep_hyper* hp, const float* z, int n_par, int n, const double* box9,
                                      const double* pos, double* e_total, double* e_atom, float* force,
                                      float* virial_atom, double* virial_total, unsigned* err_out, void* stream)
{
    if (!hp || !z || !pos) {
        set_error("nep_compute_efv_static: NULL hyperparameters, parameters or positions");
        return NEP_ERR_ARG;
    }
    if (hp->n_max_R + 1 != kNR || hp->n_max_A + 1 != kNA || hp->l_max != kLmax || hp->n_neu < 1 ||
        hp->n_neu > kMaxNeu) {
        set_error("nep_compute_efv_static: this build has kernels for n_max_R=%d, n_max_A=%d, l_max=%d, n_neu<=%d",
                  kNR - 1, kNA - 1, kLmax, kMaxNeu);
        return NEP_ERR_UNSUPPORTED;
    }
    if (!(hp->rc_R > 0.0) || !(hp->rc_A > 0.0) || n_par != (kNdes + 2) * hp->n_neu + 1) {
        set_error("nep_compute_efv_static: bad cutoffs or n_par");
        return NEP_ERR_ARG;
    }
    if (n < 1 || n > kStaticAtoms) {
        set_error("nep_compute_efv_static: n = %d atoms is outside 1..%d (the static scratch size)", n, kStaticAtoms);
        return NEP_ERR_ARG;
    }
    if (hp->max_neighbors < 1 || hp->max_neighbors > kStaticSlots) {
        set_error("nep_compute_efv_static: max_neighbors = %d is outside 1..%d (the static scratch size)",
                  hp->max_neighbors, kStaticSlots);
        return NEP_ERR_ARG;
    }
    const double rmax = hp->rc_R > hp->rc_A ? hp->rc_R : hp->rc_A;
    Box box;
    int rc = setup_box(box9, rmax, box);
    if (rc) return rc;
    const int ncell = box.nc[0] * box.nc[1] * box.nc[2];
    if (ncell > kStaticCells) {
        set_error("nep_compute_efv_static: the box needs %d cells, more than %d (the static scratch size)", ncell,
                  kStaticCells);
        return NEP_ERR_ARG;
    }
    unsigned char* base = nullptr;
    if ((rc = scratch_address(&base))) return rc;
    cudaStream_t st = (cudaStream_t)stream;

    NeighborList nl;
    nl.n_cap = kStaticAtoms;
    nl.m_cap = hp->max_neighbors;
    nl.ncell_cap = kStaticCells + 1;
    nl.count = reinterpret_cast<int*>(base + kOffCount);
    nl.nbr = reinterpret_cast<int*>(base + kOffNbr);
    nl.rev = reinterpret_cast<int*>(base + kOffRev);
    nl.pf = reinterpret_cast<float*>(base + kOffPf);
    nl.vala = reinterpret_cast<int*>(base + kOffVala);
    nl.xh = reinterpret_cast<float*>(base + kOffXh);
    nl.xl = reinterpret_cast<float*>(base + kOffXl);
    nl.atom_cell = reinterpret_cast<int*>(base + kOffAtomCell);
    nl.cell_atoms = reinterpret_cast<int*>(base + kOffCellAtoms);
    nl.cell_count = reinterpret_cast<int*>(base + kOffCellCount);
    nl.cell_start = reinterpret_cast<int*>(base + kOffCellStart);
    nl.cell_fill = reinterpret_cast<int*>(base + kOffCellFill);
    double* partials = reinterpret_cast<double*>(base + kOffPartials);
    double* red = reinterpret_cast<double*>(base + kOffRed);
    unsigned* err = reinterpret_cast<unsigned*>(base + kOffErr);

    // the cell counters and the error word must start at zero; the array
    // keeps whatever the previous call left
    if ((rc = cuda_fail(cudaMemsetAsync(nl.cell_count, 0, sizeof(int) * (ncell + 1), st), "cudaMemsetAsync")) ||
        (rc = cuda_fail(cudaMemsetAsync(nl.cell_fill, 0, sizeof(int) * (ncell + 1), st), "cudaMemsetAsync")) ||
        (rc = cuda_fail(cudaMemsetAsync(err, 0, sizeof(unsigned), st), "cudaMemsetAsync")))
        return rc;

    if ((rc = build_neighbor_list(nl, box, n, const_cast<double*>(pos), nullptr, false, nullptr, (float)rmax, err, nullptr,
                                  st)))
        return rc;
    ForceArgs fa{z, hp->n_neu, (float)hp->rc_R, (float)hp->rc_A, box};
    const int nblocks = site_blocks(n);
    double* part_e = partials;
    double* part_v = partials + ((nblocks + 7) / 8) * 8;
    int nb1 = 0, nb2 = 0, nc2 = 0;
    if ((rc = launch_site_partial_forces(fa, nl, n, e_atom, part_e, err, st, nb1))) return rc;
    AssembleArgs aa{};
    aa.rc_max = (float)rmax;
    aa.box = box;
    aa.vel = nullptr;
    if ((rc = launch_assemble(aa, nl, n, force, virial_atom, part_v, err, st, nb2, nc2))) return rc;
    if ((rc = launch_reduce(part_e, nb1, 1, red, st))) return rc;
    if ((rc = launch_reduce(part_v, nb2, nc2, red + 1, st))) return rc;
    k_static_finish<<<1, 32, 0, st>>>(red, e_total, virial_total, err, err_out);
    return cuda_fail(cudaGetLastError(), "nep_compute_efv_static kernels");
}
