// nep_internal.cuh -- shared definitions of the sm_103a NEP library.
//
// Data layout in device memory (n atoms, M = neighbour capacity per atom):
//   positions        FP64 [3][n] (caller) + FP32 hi/lo split xh, xl [n] float4
//   neighbour list   int32 nbr[M][n] = j | image_code << 24, count[n]
//                    int32 rev[M][n] = slot of i in j's list (reverse pair)
//                    int32 vala[n][M]: scratch of the list build (the rank of
//                    each unsorted slot; the values atom-major in the brute
//                    search)
//   partial forces   FP32 pf[M][n] float4 (x, y, z, unused) = dU_i/dr_ij
//                    (Eq. 23), slot-major: one 16-byte gather per reverse pair
//   forces           FP32 [3][n], per-atom virials FP32 [9][n]
// Slot-major layouts make the per-atom loops of a warp read consecutive
// addresses at every slot.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nep.h"

#ifdef __CUDA_ARCH__
#define NEP_LDG(p) __ldg(p)
#else
#define NEP_LDG(p) (*(p))
#endif

namespace nep {

__host__ __device__ __forceinline__ int imin(int a, int b) { return a < b ? a : b; }

// Packed FP32 pairs.  On the device these are the f32x2 instructions
// (__ffma2_rn / __fmul2_rn: two IEEE round-to-nearest operations per
// instruction, bitwise the same as two scalar fmaf / products); on the host
// the two scalar operations.  bcast2(x) = (x, x) is the broadcast operand.
__host__ __device__ __forceinline__ float2 bcast2(float x) { return make_float2(x, x); }

__host__ __device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c)
{
#ifdef __CUDA_ARCH__
    return __ffma2_rn(a, b, c);
#else
    return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
#endif
}

// ---------------------------------------------------------------- sizes
constexpr int kNR = 8;               // radial orders n = 0..7
constexpr int kNA = 6;               // angular radial orders n = 0..5
constexpr int kLmax = 4;             // Legendre orders l = 1..4
constexpr int kLM = 24;              // real harmonics with 1 <= l <= 4: 3+5+7+9
constexpr int kNdes = kNR + kNA * kLmax;  // 32
constexpr int kMaxNeu = 64;
constexpr int kMaxAtoms = (1 << 24) - 1;
constexpr int kImgCenter = 62;       // image code of the zero shift
// Largest cell grid of the list build (nc[0] nc[1] nc[2]).  A large, sparse
// box would otherwise need more cells than an int counts; the grid is then
// made coarser, which stays correct because every cell edge is still at
// least the list radius.
constexpr int kMaxCells = 1 << 22;

// device error word bits
enum : unsigned {
    kErrOverflow = 1u,
    kErrNonFinite = 2u,
    kErrReverse = 4u,
    kErrTimeout = 8u,
};

// Orthorhombic periodic box; lengths split into FP32 hi + lo parts so that a
// pair vector can be formed to FP32 rounding from hi/lo positions.
struct Box {
    double L[3];
    float Lh[3];
    float Ll[3];
    int nc[3];      // cells per direction (0 when the brute-force list is used)
    double cpl[3];  // cells per unit length nc / L (binning without a division)
    int img[3];     // largest |image shift| a pair can need per direction
};

// Image code of shift (sx, sy, sz), each in [-2, 2].
__host__ __device__ __forceinline__ int image_code(int sx, int sy, int sz)
{
    return (sx + 2) * 25 + (sy + 2) * 5 + (sz + 2);
}

__host__ __device__ __forceinline__ void image_shift(int code, int& sx, int& sy, int& sz)
{
    sx = code / 25 - 2;
    sy = (code / 5) % 5 - 2;
    sz = code % 5 - 2;
}

// r = (x_a + s L) - x_b from hi/lo parts.  The box length is combined first
// with whichever atom sits near the far face (b when s > 0, a when s < 0), so
// that subtraction is exact (Sterbenz) and only the final small difference
// rounds; adding L to the atom near the origin would round at ulp(L).
__host__ __device__ __forceinline__ float diff1(float ah, float al, float bh, float bl, float s, float Lh, float Ll)
{
    const float hi = (s > 0.f) ? ah - fmaf(-s, Lh, bh) : fmaf(s, Lh, ah) - bh;
    const float lo = fmaf(s, Ll, al - bl);
    return hi + lo;
}

// Pair vector r_ij = x_j + shift(code) - x_i, evaluated in a canonical
// orientation so that r_ji == -r_ij bit for bit.  Both atoms' hi/lo
// coordinates are passed in.
__host__ __device__ __forceinline__ void pair_vector(int i, int j, int code, const float (&hi)[3], const float (&li)[3],
                                            const float (&hj)[3], const float (&lj)[3], const Box& b, float& rx,
                                            float& ry, float& rz)
{
    int sx, sy, sz;
    image_shift(code, sx, sy, sz);
    const bool fwd = (j > i) || (j == i && code < kImgCenter);
    const float sg = fwd ? 1.f : -1.f;
    const float fx = fwd ? (float)sx : (float)(-sx);
    const float fy = fwd ? (float)sy : (float)(-sy);
    const float fz = fwd ? (float)sz : (float)(-sz);
    // a = the atom whose image is shifted, b = the origin atom
    rx = sg * diff1(fwd ? hj[0] : hi[0], fwd ? lj[0] : li[0], fwd ? hi[0] : hj[0], fwd ? li[0] : lj[0], fx, b.Lh[0],
                    b.Ll[0]);
    ry = sg * diff1(fwd ? hj[1] : hi[1], fwd ? lj[1] : li[1], fwd ? hi[1] : hj[1], fwd ? li[1] : lj[1], fy, b.Lh[1],
                    b.Ll[1]);
    rz = sg * diff1(fwd ? hj[2] : hi[2], fwd ? lj[2] : li[2], fwd ? hi[2] : hj[2], fwd ? li[2] : lj[2], fz, b.Lh[2],
                    b.Ll[2]);
}

// pair_vector that also returns the rounding residual of each component:
// r_exact = r + r_lo to within the tiny rounding of the lo parts (~1e-14 A).
// The hi-part difference is exact, so r = hi + lo rounds once and Fast2Sum
// recovers what that rounding dropped.
__host__ __device__ __forceinline__ float diff1_lo(float ah, float al, float bh, float bl, float s, float Lh, float Ll,
                                                   float& r_lo)
{
    const float hi = (s > 0.f) ? ah - fmaf(-s, Lh, bh) : fmaf(s, Lh, ah) - bh;
    const float lo = fmaf(s, Ll, al - bl);
    const float r = hi + lo;
    r_lo = lo - (r - hi);
    return r;
}

__host__ __device__ __forceinline__ void pair_vector_lo(int i, int j, int code, const float (&hi)[3],
                                                        const float (&li)[3], const float (&hj)[3],
                                                        const float (&lj)[3], const Box& b, float (&r)[3],
                                                        float (&r_lo)[3])
{
    int sx, sy, sz;
    image_shift(code, sx, sy, sz);
    const bool fwd = (j > i) || (j == i && code < kImgCenter);
    const float sg = fwd ? 1.f : -1.f;
    const float f[3] = {fwd ? (float)sx : (float)(-sx), fwd ? (float)sy : (float)(-sy),
                        fwd ? (float)sz : (float)(-sz)};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float rl;
        r[d] = sg * diff1_lo(fwd ? hj[d] : hi[d], fwd ? lj[d] : li[d], fwd ? hi[d] : hj[d], fwd ? li[d] : lj[d], f[d],
                             b.Lh[d], b.Ll[d], rl);
        r_lo[d] = sg * rl;
    }
}

// FP32 hi/lo positions are stored as one float4 record (x, y, z, 0) per atom
// for each part, so a neighbour's coordinates arrive in two 16-byte loads.
__host__ __device__ __forceinline__ void load_pos(const float* __restrict__ xh, const float* __restrict__ xl, int n, int i,
                                         float (&h)[3], float (&l)[3])
{
    (void)n;
    const float4 a = NEP_LDG(reinterpret_cast<const float4*>(xh) + i);
    const float4 b = NEP_LDG(reinterpret_cast<const float4*>(xl) + i);
    h[0] = a.x;
    h[1] = a.y;
    h[2] = a.z;
    l[0] = b.x;
    l[1] = b.y;
    l[2] = b.z;
}


// Split an FP64 value into FP32 hi + lo.
__host__ __device__ __forceinline__ void split_hilo(double x, float& h, float& l)
{
    h = (float)x;
    l = (float)(x - (double)h);
}

// The hi record's fourth word carries the atom's species number Z (1 for a
// single species): the multicomponent weighting f_c -> f_c sqrt(Z_i Z_j).
__host__ __device__ __forceinline__ void store_pos(float* __restrict__ xh, float* __restrict__ xl, int i, const double (&x)[3],
                                                  float zi = 1.f)
{
    float h[3], l[3];
    for (int d = 0; d < 3; ++d) split_hilo(x[d], h[d], l[d]);
    reinterpret_cast<float4*>(xh)[i] = make_float4(h[0], h[1], h[2], zi);
    reinterpret_cast<float4*>(xl)[i] = make_float4(l[0], l[1], l[2], 0.f);
}

__host__ __device__ __forceinline__ float load_z(const float* __restrict__ xh, int i)
{
    return reinterpret_cast<const float4*>(xh)[i].w;
}

// Warp sum of K <= 16 doubles held by every lane.  Each butterfly level keeps
// half of the remaining components (the lane sends the half its partner keeps),
// so a lane does 8 + 4 + 2 + 1 + 1 additions instead of 5 K.  On return
// lanes 2c and 2c + 1 hold the warp total of component warp_comp(lane) (the
// pattern is fixed, so the sums are deterministic).
__device__ __forceinline__ int warp_comp(int lane)
{
    return ((lane & 16) ? 8 : 0) + ((lane & 8) ? 4 : 0) + ((lane & 4) ? 2 : 0) + ((lane & 2) ? 1 : 0);
}

template <int K>
__device__ __forceinline__ double warp_sum_multi(const double (&v)[K])
{
    static_assert(K <= 16, "at most 16 components");
    const int lane = threadIdx.x & 31;
    double a[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) a[c] = c < K ? v[c] : 0.0;
#pragma unroll
    for (int h = 8, o = 16; h >= 1; h >>= 1, o >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int c = 0; c < h; ++c) {
            const double send = upper ? a[c] : a[c + h];
            const double keep = upper ? a[c + h] : a[c];
            a[c] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return a[0] + __shfl_xor_sync(0xffffffffu, a[0], 1);
}

// Block-wide sum of K doubles; thread 0 writes out[k].  blockDim.x must be a
// multiple of 32 and at most 1024.
template <int K>
__device__ __forceinline__ void block_sum_store(double (&v)[K], double* __restrict__ out)
{
    __shared__ double red[32][K];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    if constexpr (K >= 4) {
        const double s = warp_sum_multi<K>(v);
        const int c = warp_comp(lane);
        if ((lane & 1) == 0 && c < K) red[warp][c] = s;
        __syncthreads();
        if (warp == 0) {
            double w[K];
#pragma unroll
            for (int k = 0; k < K; ++k) w[k] = lane < nw ? red[lane][k] : 0.0;
            const double t = warp_sum_multi<K>(w);
            if ((lane & 1) == 0 && c < K) out[c] = t;
        }
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < K; ++k) red[warp][k] = v[k];
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                double s = lane < nw ? red[lane][k] : 0.0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) out[k] = s;
            }
        }
    }
}

// ---------------------------------------------------------------- workspace
struct NeighborList {
    int n_cap = 0;       // atoms the buffers hold
    int m_cap = 0;       // neighbour slots per atom
    int ncell_cap = 0;
    int* count = nullptr;
    int* nbr = nullptr;
    int* rev = nullptr;
    int* vala = nullptr;     // list-build scratch [n][m_cap] (slot ranks, or values atom-major)
    float* pf = nullptr;
    float* xh = nullptr;
    float* xl = nullptr;
    int* atom_cell = nullptr;
    int* cell_count = nullptr;
    int* cell_start = nullptr;
    int* cell_fill = nullptr;
    int* cell_atoms = nullptr;
    // [3][n] words: bit k of atom i set when slot k lies within the cutoff,
    // written by the site pass when it compacts its staged slots; `mask_set`
    // (host) says whether the last site pass launched wrote them, so that
    // the assembly skips the other slots' loads.
    unsigned* mask = nullptr;
    bool mask_set = false;
};

struct Workspace {
    NeighborList nl;
    double* partials = nullptr;  // per-block FP64 partial sums
    int partial_cap = 0;         // doubles
    float* force = nullptr;      // [3][n] FP32 (MD and internal use)
    int force_cap = 0;
    float* plain = nullptr;      // [2][32][n] q and G of the plain comparator (on demand)
    int plain_cap = 0;
};

// host-side helpers (nep_api.cu)
void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
int ensure_workspace(Workspace& ws, int n, int m_cap, int ncell, int nblocks_partials);
void free_workspace(Workspace& ws);
int setup_box(const double* box9, double r_list, Box& b);

// neighbour list (nep_neighbor.cu)
// mode: build from positions `pos` (FP64 [3][n]); when wrap_in_place is true
// the wrapped positions are written back to pos and to x_ref (if non-null).
// zatom: species number of every atom (dev [n]) or NULL (all 1)
int build_neighbor_list(NeighborList& nl, const Box& b, int n, double* pos, const float* zatom, bool wrap_in_place,
                        double* x_ref,
                        float r_list, unsigned* d_err, const unsigned* d_gate, cudaStream_t st);

// force path (nep_force.cu)
struct ForceArgs {
    const float* z;          // parameters on the device
    int n_neu;
    float rcR, rcA;
    Box box;
    int typed = 0;           // species numbers in the position records are used (multicomponent)
    int nr = kNR;            // radial orders n_max^R + 1 (8, or 13 for the split model)
    int na = kNA;            // angular radial orders n_max^A + 1 (6, or 7)
};
// The descriptor sizes with force-path kernels: the 32-descriptor model
// (n_max^R = 7, n_max^A = 5) and the split 41-descriptor model (12, 6),
// both with l_max = 4.  Only the force path (energies, forces, virials, MD)
// has kernels for the second; training sets, the plain comparator and the
// allocation-free call need the first.
inline bool sizes_default(const nep_hyper& h) { return h.n_max_R == kNR - 1 && h.n_max_A == kNA - 1; }
inline bool sizes_split(const nep_hyper& h) { return h.n_max_R == 12 && h.n_max_A == 6; }
// the site pass runs kSiteAtomsPerBlock atoms per block; its per-block
// energy partials need site_blocks(n) slots, which also bounds the block
// counts of the assembly and of the plain comparator
constexpr int kSiteAtomsPerBlock = 128;
inline int site_blocks(int n) { return (n + kSiteAtomsPerBlock - 1) / kSiteAtomsPerBlock; }
int launch_site_partial_forces(const ForceArgs& a, NeighborList& nl, int n, double* e_atom, double* e_partials,
                               unsigned* d_err, cudaStream_t st, int& nblocks);
struct AssembleArgs {
    float rc_max;
    Box box;
    // MD extras (used when vel != nullptr)
    double* vel;
    double half_dt_over_m;   // dt/2 / (m * unit)
    double ke_factor;        // 0.5 m * unit
    bool heat;
};
int launch_assemble(const AssembleArgs& a, NeighborList& nl, int n, float* force, float* virial_atom,
                    double* partials, unsigned* d_err, cudaStream_t st, int& nblocks, int& ncomp);
int launch_reduce(const double* partials, int nblocks, int ncomp, double* out, cudaStream_t st);
// the plain FP32 comparator (nep_plain.cu): descriptors, network and partial
// forces by the literal formulas, q and G [32][n] scratch
int launch_plain_site(const ForceArgs& a, NeighborList& nl, int n, float* q, float* G, double* e_atom,
                      double* e_partials, unsigned* d_err, cudaStream_t st, int& nblocks);

}  // namespace nep

namespace nep {
// CUDA-event pairs around kernel launches (enabled on demand).
struct Profiler {
    bool on = false;
    struct Slot {
        cudaEvent_t a = nullptr, b = nullptr;
        int kind = 0;
    };
    Slot* slots = nullptr;
    int cap = 0, used = 0;
    // returns the slot to bracket a launch of `kind`, or nullptr when off/full
    Slot* begin(int kind, cudaStream_t st);
    void end(Slot* s, cudaStream_t st);
    int read(double* ms, long long* cnt);  // ms[NEP_PROFILE_KINDS], cnt[...]; synchronises
    void release();
};
// tensor-core population network (nep_pop_tc.cu)
size_t pop_tc_packed_bytes(int P);
// kernel attributes of the tensor-core path; call outside any stream capture
int prepare_pop_tc();
// G [N][32][Pst] FP32, U [N][P] FP64 (launches only: capturable)
// the descriptors packed as split-BF16 GEMM-1 A tiles, once per training set
size_t pop_tc_qpack_bytes(int N);
int launch_pack_q_tc(int N, const float* q, unsigned char* qpack, cudaStream_t st);
// Layout of G written by the population network:
//   kGRowsF32  [N][32][Pst] FP32;   kGRowsF16  [N][32][Pst] FP16;
//   kGTilesF16 per atom the tensor-core B tile of the owner pass: members
//              as rows of a K-major [8 ceil(Pst / 8)] x 32 FP16 tile
//              (owner_tc_g_bytes(Pst) bytes per atom, nep_tc.cuh layout).
enum GLayout { kGRowsF32 = 0, kGRowsF16 = 1, kGTilesF16 = 2 };
// z: the population [P][n_par] (packed into the group records by the launch),
// or NULL when `packed` already holds it (launch_pack_tc_draw)
// pipelined: the persistent warp-specialised kernel (same bits), else one CTA
// per (member group, 128-atom tile)
int launch_pop_tc(int N, int P, int Pst, int n_neu, const unsigned char* qpack, const float* z, unsigned char* packed,
                  void* G, int g_layout, double* U, unsigned* err, bool pipelined, cudaStream_t st);
// An SNES generation's draws and population packed in one launch: r [P][n_par]
// the standard normals of generation *d_gen (the stream of nep_philox.cuh),
// z = m + s (.) r, and the group records of z, with the same bits as the draw
// kernel followed by the packing of launch_pop_tc.
int launch_pack_tc_draw(int P, int n_neu, unsigned long long seed, const unsigned* d_gen, const float* m,
                        const float* s, float* r, float* z, unsigned char* packed, cudaStream_t st);

// The first contraction pass on the tensor cores (BF16 precision mode).  A
// tile is up to 128 rows of one owner atom j: three per pair (the Jacobian
// rows d p / d G of components x, y, z), and in the owner's first tile three
// rows of its own term (B_j) and six of its virial contribution
// (-sum_pairs r^a J^b, components xx yy zz xy yz zx).
struct OwnerTile {
    int j;           // owner atom
    int nt;          // pairs in this tile
    int extra;       // 1: the own-term and virial rows follow the pair rows
    int groups;      // 8-row groups stored
    long long q0;    // first pair (owner order)
    long long row0;  // first row of the tile in the packed operand (multiple of 8)
};
constexpr int kOwnerTcPairs = 39;  // pairs of a first tile (3 x 39 + 9 <= 128 rows)
constexpr int kOwnerTcMorePairs = 42;  // pairs of each further tile
// bytes of one atom's G tile in the kGTilesF16 layout
__host__ __device__ inline size_t owner_tc_g_bytes(int Pst) { return (size_t)((Pst + 7) / 8) * 512; }
struct PairRec;
// packs the Jacobian rows of every tile as FP16 (each row scaled by a power
// of two, kept in rowscale, so that its largest entry lies in [2^13, 2^14));
// once per training set
int launch_pack_owner_tc(int n_tiles, const OwnerTile* tiles, const PairRec* rec, const long long* aidx,
                         const float* ang, const float* B, const long long* pstart, unsigned char* apack,
                         float* rowscale, cudaStream_t st);
int prepare_owner_tc();
// tiles [t0, t1): partial forces p_kji (FP16, at the receiver's slot rev[q]),
// own terms and virial terms (FP32), as the CUDA-core owner pass writes them
int launch_owner_tc(int t0, int t1, const OwnerTile* tiles, const unsigned char* apack, const float* rowscale,
                    const void* G, int Pst, const long long* rev, void* pbuf, float* fown, float* w6, unsigned* err,
                    cudaStream_t st);

}  // namespace nep

struct nep_model {
    nep_hyper hp;
    nep::Profiler prof;
    int n_des = 0;
    int n_par = 0;
    float* d_z = nullptr;
    unsigned* d_err = nullptr;   // latched device error bits
    double* d_red = nullptr;     // reduction outputs (32 doubles)
    nep::Workspace ws;
    float* zatom = nullptr;      // species numbers of the atoms (nep_set_species), or NULL
    int zatom_n = 0;
};

namespace nep {
// status from latched device error bits
int status_from_bits(unsigned bits);
}
