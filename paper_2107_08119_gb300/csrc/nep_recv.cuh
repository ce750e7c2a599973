// nep_recv.cuh -- device helpers of the SNES receiver pass (the second
// contraction pass: F_i = G_i . B_i - sum_j p_kji, and the per-chunk loss sums
// of Eqs. 30-32), used by the receiver kernels of nep_train.cu; nep_pop_tc.cu
// takes the population bound kMaxPop from here.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include "nep_internal.cuh"
#include "nep_tc.cuh"

namespace nep {
namespace {

constexpr int kMaxPop = 64;

// Partial-force element loads: FP32, or FP16 in the BF16 precision mode; two
// members at a time.
__device__ __forceinline__ float2 pb_load2(const float* o) { return *reinterpret_cast<const float2*>(o); }
__device__ __forceinline__ float2 pb_load2(const __half* o)
{
    return __half22float2(*reinterpret_cast<const __half2*>(o));
}

constexpr int kReceiverThreads = 256;

__device__ __forceinline__ void discard_l2_lines(const void* lo, const void* hi, int lane)
{
    const uintptr_t a = ((uintptr_t)lo + 127) & ~(uintptr_t)127, b = (uintptr_t)hi & ~(uintptr_t)127;
    for (uintptr_t l = a + (uintptr_t)lane * 128; l < b; l += 32 * 128)
        asm volatile("discard.global.L2 [%0], 128;" ::"l"(l) : "memory");
}

// Per-atom operands of the receiver pass, loaded one atom ahead.
struct RecvAtom {
    float2 fo[3];         // G_i . B_i of the lane's two members
    float2 w6[6];         // owner virial terms
    double u0, u1;        // site energies
    float t[3];           // F_tar
    long long ps, pe;     // slot range
};

// The own and virial terms are read through L2 (ld.global.cg, no L1
// allocation): each is read once.
__device__ __forceinline__ void recv_load(RecvAtom& a, int i, int P, int Pst, int k0, bool ld, bool on0, bool on1,
                                          const double* __restrict__ U, const long long* __restrict__ pstart,
                                          const float* __restrict__ fown, const float* __restrict__ w6in,
                                          const float* __restrict__ f_tar)
{
    const float* o = fown + (size_t)i * 3 * Pst + k0;
    const float* w = w6in + (size_t)i * 6 * Pst + k0;
#pragma unroll
    for (int c = 0; c < 3; ++c)
        a.fo[c] = ld ? __ldcg(reinterpret_cast<const float2*>(o + (size_t)c * Pst)) : make_float2(0.f, 0.f);
#pragma unroll
    for (int c = 0; c < 6; ++c)
        a.w6[c] = ld ? __ldcg(reinterpret_cast<const float2*>(w + (size_t)c * Pst)) : make_float2(0.f, 0.f);
    a.u0 = on0 ? U[(size_t)i * P + k0] : 0.0;
    a.u1 = on1 ? U[(size_t)i * P + k0 + 1] : 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) a.t[c] = f_tar[(size_t)i * 3 + c];
    a.ps = pstart[i];
    a.pe = pstart[i + 1];
}

// A warp's running sums over its atoms of one chunk, for the lane's two
// members: U in FP64 (site energies come as FP64), the squared force
// residuals and the owner virial terms in FP32 (a warp takes at most
// kChunkAtoms / 8 = 4 atoms of a chunk; the FP64 pipe is slow on this part, so
// the per-atom terms stay off it), converted once per chunk to FP64.
struct RecvAcc {
    double u[2] = {0.0, 0.0};
    float f[2] = {0.f, 0.f};
    float w[2][6] = {{0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}};
    __device__ __forceinline__ void add(const RecvAtom& a, const float (&F)[2][3])
    {
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const float dx = F[m][0] - a.t[0], dy = F[m][1] - a.t[1], dz = F[m][2] - a.t[2];
            u[m] += m == 0 ? a.u0 : a.u1;
            f[m] += fmaf(dz, dz, fmaf(dy, dy, dx * dx));
#pragma unroll
            for (int c = 0; c < 6; ++c) w[m][c] += m == 0 ? a.w6[c].x : a.w6[c].y;
        }
    }
    // the lane's rows of the warp's slice (members past kMaxPop have none)
    __device__ __forceinline__ void store(double* ru, float (*rf)[7], int k0) const
    {
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            if (k0 + m >= kMaxPop) continue;
            ru[k0 + m] = u[m];
            rf[k0 + m][0] = f[m];
#pragma unroll
            for (int c = 0; c < 6; ++c) rf[k0 + m][1 + c] = w[m][c];
        }
    }
};

// The loss partials of one chunk and member (64 bytes): the sum of U in
// FP64, then the squared force residuals and the six owner virial sums in
// FP32, as the receiver forms them (the loss kernel adds them in FP32 too:
// the FP64 pipe is slow on this part).
struct ChunkRec {
    double u;
    float fw[7];  // |F - F_tar|^2, W_xx, W_yy, W_zz, W_xy, W_yz, W_zx
    float pad[7];
};
static_assert(sizeof(ChunkRec) == 64, "one record is eight FP64 slots of the partials buffer");

// Per-warp sums of a receiver block: U in FP64, the other seven terms in FP32.
template <int W>
struct RecvRed {
    double u[W][kMaxPop];
    float f[W][kMaxPop][7];
};

// The chunk's partials in a fixed order (warps 0..W-1): U summed in FP64,
// the squared force residuals and virial terms in FP32.  partials: the
// buffer of ChunkRec records [chunk][member], this chunk's P records.
template <int W>
__device__ __forceinline__ void recv_chunk_store(const RecvRed<W>& red, int P, double* __restrict__ partials)
{
    ChunkRec* out = reinterpret_cast<ChunkRec*>(partials);
    for (int e = threadIdx.x; e < P * 8; e += blockDim.x) {
        const int k = e / 8, w = e % 8;
        if (w == 0) {
            double a = 0.0;
#pragma unroll
            for (int q = 0; q < W; ++q) a += red.u[q][k];
            out[k].u = a;
        } else {
            float a = 0.f;
#pragma unroll
            for (int q = 0; q < W; ++q) a += red.f[q][k][w - 1];
            out[k].fw[w - 1] = a;
        }
    }
}

// The receiver pass with each atom's slot rows brought into shared memory by
// bulk asynchronous copies (cp.async.bulk, completion counted on an
// mbarrier).  A receiver's slots are contiguous in the partial-force buffer,
// so lane 0 of a warp requests them as pieces of at most kBulkStage bytes,
// two pieces ahead of the lanes' sums (two buffers per warp); a piece's
// first and last bytes are rounded out to 16-byte boundaries (the buffer is
// allocated in FP32 units, so in FP16 mode the rounded end stays inside it;
// FP32 slots are multiples of 48 bytes and need no rounding).  The lanes add
// from shared memory in slot order: the same atoms per warp, terms and order
// of summation as k_contract, hence the same bits.  Every wait is bounded: a
// copy that does not land latches NEP_ERR_TIMEOUT and the warp stops summing;
// it then waits (bounded) for its copies still in flight before the block
// exits, so no copy writes into shared memory another block owns.
constexpr int kBulkStage = 4096;           // payload bytes of one piece
constexpr int kBulkBuf = kBulkStage + 32;  // + the rounding at both ends (16-byte multiple)
constexpr int kBulkSmem = (kReceiverThreads / 32) * 2 * kBulkBuf;
constexpr uint32_t kBulkPolls = 1u << 22;

// Per-warp state of the bulk receiver kept across chunks: the pieces issued
// to and waited on its two mbarriers (piece n: buffer n & 1, phase parity
// (n >> 1) & 1).
struct BulkWarp {
    unsigned issued = 0u, waited = 0u;
};

// Shared memory of the bulk receiver: per warp two piece buffers and two
// mbarriers (initialised once by bulk_init), and the warps' sums.
struct BulkSmem {
    unsigned char buf[kReceiverThreads / 32][2][kBulkBuf];
    uint64_t bar[kReceiverThreads / 32][2];
    RecvRed<kReceiverThreads / 32> red;
};

__device__ __forceinline__ void bulk_init(BulkSmem& S)
{
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        tc::mbar_init(&S.bar[warp][0], 1);
        tc::mbar_init(&S.bar[warp][1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
}

// The receiver work of chunk c, by all kReceiverThreads threads of the block
// (it ends with a block barrier): every atom's F_i from its slot rows, summed
// in slot order, and the chunk's partials (recv_chunk_store).  With
// `discard`, the 128-byte L2 lines lying wholly inside an atom's slot rows are
// dropped once they have landed in shared memory (no write-back of rows that
// the next evaluation rewrites).  Returns false if a copy did not land in
// time (NEP_ERR_TIMEOUT is latched); the caller then drains with bulk_drain
// before its shared memory goes.
template <class PT>
__device__ bool bulk_receive_chunk(int c, int P, int Pst, const int* __restrict__ chunk_begin,
                                   const int* __restrict__ chunk_end, const double* __restrict__ U,
                                   const long long* __restrict__ pstart, const float* __restrict__ fown,
                                   const PT* __restrict__ pbuf, const float* __restrict__ w6in,
                                   const float* __restrict__ f_tar, double* __restrict__ partials,
                                   unsigned* __restrict__ err, bool discard, BulkSmem& S, BulkWarp& bw)
{
    constexpr int kWarps = kReceiverThreads / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k0 = 2 * lane;
    const bool on0 = k0 < P, on1 = k0 + 1 < P;
    const bool ld = k0 < Pst;
    const long long slot_bytes = 3LL * Pst * (long long)sizeof(PT);
    const long long per_piece = kBulkStage / slot_bytes;  // >= 5 slots (Pst <= 64)
    const unsigned char* src = reinterpret_cast<const unsigned char*>(pbuf);
    RecvAcc acc;
    const int end = chunk_end[c];
    // producer cursor: atom pa, its next slot pp and its slot end pend
    int pa = chunk_begin[c] + warp;
    long long pp = 0, pend = 0;
    if (pa < end) {
        pp = pstart[pa];
        pend = pstart[pa + 1];
    }
    // requests the next piece of this warp's atoms, if any
    auto issue = [&]() {
        while (pa < end && pp >= pend) {
            pa += kWarps;
            if (pa < end) {
                pp = pstart[pa];
                pend = pstart[pa + 1];
            }
        }
        if (pa >= end) return;
        const long long q1 = min(pend, pp + per_piece);
        const size_t b0 = (size_t)(pp * slot_bytes), b1 = (size_t)(q1 * slot_bytes);
        const size_t a0 = b0 & ~(size_t)15, a1 = (b1 + 15) & ~(size_t)15;
        const int s = (int)(bw.issued & 1u);
        if (lane == 0) {
            const uint32_t bb = tc::smem_u32(&S.bar[warp][s]);
            // the buffer's previous piece was read by ordinary loads (ordered by the __syncwarp before this call)
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bb), "r"((uint32_t)(a1 - a0))
                         : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                             tc::smem_u32(S.buf[warp][s])),
                         "l"(src + a0), "r"((uint32_t)(a1 - a0)), "r"(bb)
                         : "memory");
        }
        pp = q1;
        ++bw.issued;
    };
    issue();
    issue();
    bool ok = true;
    int i = chunk_begin[c] + warp;
    RecvAtom cur, nxt;
    if (i < end) recv_load(cur, i, P, Pst, k0, ld, on0, on1, U, pstart, fown, w6in, f_tar);
    for (; ok && i < end; i += kWarps) {
        if (i + kWarps < end) recv_load(nxt, i + kWarps, P, Pst, k0, ld, on0, on1, U, pstart, fown, w6in, f_tar);
        float F[2][3] = {{cur.fo[0].x, cur.fo[1].x, cur.fo[2].x}, {cur.fo[0].y, cur.fo[1].y, cur.fo[2].y}};
        for (long long q0 = cur.ps; q0 < cur.pe; q0 += per_piece) {
            const long long q1 = min(cur.pe, q0 + per_piece);
            const int s = (int)(bw.waited & 1u);
            ok = __all_sync(0xffffffffu, tc::mbar_wait(&S.bar[warp][s], (bw.waited >> 1) & 1u, kBulkPolls));
            if (!ok) break;
            ++bw.waited;
            const size_t b0 = (size_t)(q0 * slot_bytes);
            const unsigned char* base = S.buf[warp][s] + (b0 - (b0 & ~(size_t)15));
            if (ld)
                for (long long q = q0; q < q1; ++q) {
                    const PT* o = reinterpret_cast<const PT*>(base + (size_t)((q - q0) * slot_bytes)) + k0;
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc) {
                        const float2 x = pb_load2(o + (size_t)cc * Pst);
                        F[0][cc] -= x.x;
                        F[1][cc] -= x.y;
                    }
                }
            __syncwarp();  // every lane has read the buffer before it is refilled
            issue();
        }
        if (!ok) break;
        if (discard) discard_l2_lines(pbuf + (size_t)cur.ps * 3 * Pst, pbuf + (size_t)cur.pe * 3 * Pst, lane);
        acc.add(cur, F);
        cur = nxt;
    }
    if (!ok && lane == 0) atomicOr(err, kErrTimeout);
    acc.store(S.red.u[warp], S.red.f[warp], k0);
    __syncthreads();
    recv_chunk_store(S.red, P, partials + (size_t)c * P * 8);
    __syncthreads();  // the sums are read before the next chunk writes them
    return __syncthreads_and(ok) != 0;
}

// After a failed chunk: the warp's copies still in flight land before the
// block's shared memory goes (bounded).
__device__ __forceinline__ void bulk_drain(BulkSmem& S, BulkWarp& bw)
{
    const int warp = threadIdx.x >> 5;
    for (; bw.waited < bw.issued; ++bw.waited)
        tc::mbar_wait(&S.bar[warp][bw.waited & 1u], (bw.waited >> 1) & 1u, kBulkPolls);
}

}  // namespace
}  // namespace nep
