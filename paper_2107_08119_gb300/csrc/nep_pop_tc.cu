// nep_pop_tc.cu -- the SNES population network on the tensor cores (sm_103a).
//
// For a population of P parameter vectors z_k and all N training atoms, the
// network of Eqs. 21-22 and its input gradient are two dense contractions:
//   H[i, (k, mu)] = sum_nu q_i,nu w1_k,mu,nu            (GEMM 1, K = 32)
//   x = tanh(H - b1), U_ki = sum_mu w2_k,mu x - b2_k,  D_ki,mu = w2_k,mu (1 - x^2)
//   G_k[i, nu] = sum_mu D_ki,mu w1_k,mu,nu              (GEMM 2 per member, K = 30 -> 32)
// One CTA owns 128 atoms and one group of 4 members (grid: tiles x groups):
// GEMM 1 fills 4 x 32 TMEM columns (neurons padded to 32 per member), the
// epilogue turns them into U and D, and GEMM 2 writes G of the 4 members back
// into the same 128 columns.  Operands are split BF16 (hi + lo) in shared
// memory (canonical K-major layout, nep_tc.cuh); accumulation is FP32 in
// TMEM.  One thread issues the MMAs and commits them to an mbarrier; all
// waits are bounded (a timeout is latched as an error and the CTA still frees
// its TMEM).  G is written as [N][32][Pst]: each thread stores its atom's 16
// descriptors x 4 members as 16-byte pieces.
#include <cuda_bf16.h>

#include "nep_internal.cuh"
#include "nep_tc.cuh"

namespace nep {
namespace {

constexpr uint32_t kMaxPolls = 1u << 22;
constexpr int kTile = 128;       // atoms per CTA (TMEM lanes)
constexpr int kPopThreads = 256; // two warps per TMEM lane quarter

__device__ __forceinline__ void put_bf16(unsigned char* base, int row, int k, float v)
{
    *reinterpret_cast<__nv_bfloat16*>(base + tc::kmajor_offset(row, k)) = __float2bfloat16_rn(v);
}

// ----------------------------------------------------------------- self-test
// D (128 x N, FP32, row-major) = A (128 x 32 BF16 row-major) * B^T (B: N x 32
// BF16 row-major), one tile, N a multiple of 16 in [16, 256].
__global__ void __launch_bounds__(128) k_tc_selftest(const __nv_bfloat16* __restrict__ A,
                                                     const __nv_bfloat16* __restrict__ B, int N,
                                                     float* __restrict__ D, unsigned* err)
{
    __shared__ __align__(1024) unsigned char sA[kTile * 64];
    __shared__ __align__(1024) unsigned char sB[256 * 64];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int t = threadIdx.x, warp = t >> 5;
    for (int k = 0; k < 32; ++k)
        *reinterpret_cast<__nv_bfloat16*>(sA + tc::kmajor_offset(t, k)) = A[t * 32 + k];
    for (int r = t; r < N; r += blockDim.x)
        for (int k = 0; k < 32; ++k) *reinterpret_cast<__nv_bfloat16*>(sB + tc::kmajor_offset(r, k)) = B[r * 32 + k];
    if (t == 0) {
        tc::mbar_init(&mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        tc::tmem_alloc(&tmem_base, 256);
        tc::tmem_relinquish();
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tb = tmem_base;
    if (t == 0) {
        const uint32_t idesc = tc::idesc_bf16_f32(kTile, N);
        for (int ks = 0; ks < 2; ++ks)
            tc::mma_bf16(tb, tc::smem_desc(tc::smem_u32(sA) + ks * 256, 128, 512),
                         tc::smem_desc(tc::smem_u32(sB) + ks * 256, 128, 512), idesc, ks > 0);
        tc::mma_commit(&mbar);
    }
    const bool ok = __syncthreads_and(tc::mbar_wait(&mbar, 0, kMaxPolls)) != 0;
    if (!ok && (t & 31) == 0) atomicOr(err, kErrTimeout);
    tc::fence_after_sync();
    if (ok) {
        for (int c0 = 0; c0 < N; c0 += 8) {
            uint32_t r[8];
            tc::tmem_ld8(tb + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
            tc::tmem_ld_wait();
#pragma unroll
            for (int q = 0; q < 8; ++q) D[(size_t)t * N + c0 + q] = __uint_as_float(r[q]);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tb, 256);
}

// ----------------------------------------------------------------- population
// Members go in groups of kGroup = 4.  Per group the operands are packed once
// per evaluation (k_pack_tc) in the exact shared-memory layout, as split BF16
// pairs hi + lo with hi = bf16(x), lo = bf16(x - hi).  GEMM 1 (which sets the
// site energies) takes three MMAs, hi*hi + hi*lo + lo*hi, carrying ~16
// mantissa bits instead of 8; GEMM 2 (forces, whose loss terms average the
// rounding out) keeps D in BF16 and splits only W1 (two MMAs).  Every MMA is
// BF16 x BF16 -> FP32.  GEMM-1 columns are 32 per member (neurons past n_neu
// have zero weights), so every member starts on an 8-column TMEM boundary.
constexpr int kTcGroup = 4;
constexpr int kW1Bytes = kTile * 64;     // GEMM-1 B: 128 rows (32 m + mu) x 32 nu
constexpr int kW1tBytes = 32 * 64;       // GEMM-2 B per member: 32 nu x 32 mu
constexpr int kTileBytes = kTile * 64;   // one 128 x 32 BF16 operand tile
// packed group record: w1 hi, w1 lo, w1t hi[4], w1t lo[4], b1[4][32], w2[4][32], b2[4]
constexpr int kGroupBytes = 2 * kW1Bytes + 2 * kTcGroup * kW1tBytes + (2 * kTcGroup * 32 + 4) * 4;
constexpr int kTmemCols = 128;

// Shared memory of one CTA (one 128-atom tile, one member group).  The
// descriptor tiles and the group record arrive by bulk async copies
// (cp.async.bulk, completion counted on mbar_ld).  Once GEMM 1 has completed its operands are dead and the GEMM-2 A
// tiles (D of the four members, BF16) take their place:
//   a    q hi | q lo            -> D of members 0 | 1
//   grp  w1 hi | w1 lo | ...    -> D of members 2 | 3 | (w1t hi, w1t lo, b1, w2, b2 kept)
// ~50 KB and 128 TMEM columns per CTA: four CTAs fit on one SM.
struct PopSmem {
    unsigned char a[2 * kTileBytes];
    unsigned char grp[kGroupBytes];
    uint64_t mbar;     // MMA completion (phases 0 and 1)
    uint64_t mbar_ld;  // bulk copy of the group record
    uint32_t tmem_base;
};
static_assert(kGroupBytes % 16 == 0, "the group record is copied in 16-byte units");

__device__ __forceinline__ unsigned char* d_tile(PopSmem& S, int m)
{
    return m < 2 ? S.a + m * kTileBytes : S.grp + (m - 2) * kTileBytes;
}

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo)
{
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b)
{
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

__device__ __forceinline__ void put_split(unsigned char* hi_base, unsigned char* lo_base, int row, int k, float v)
{
    __nv_bfloat16 h, l;
    split_bf16(v, h, l);
    const uint32_t o = tc::kmajor_offset(row, k);
    *reinterpret_cast<__nv_bfloat16*>(hi_base + o) = h;
    *reinterpret_cast<__nv_bfloat16*>(lo_base + o) = l;
}

// The descriptors of every 128-atom tile as the GEMM-1 A operand, split BF16
// (hi tile, then lo tile, canonical K-major layout; rows past N are zero):
// one thread per (atom row, 8 descriptors).  Run once per training set.
__global__ void k_pack_q_tc(int N, int tiles, const float* __restrict__ q, unsigned char* __restrict__ qpack)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= tiles * kTile * 4) return;
    const int tile = e / (kTile * 4), row = (e / 4) % kTile, c = e % 4;
    const int i = tile * kTile + row;
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = i < N ? q[(size_t)i * kNdes + 8 * c + k] : 0.f;
    uint32_t h[4], l[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        __nv_bfloat16 h0, l0, h1, l1;
        split_bf16(v[2 * k], h0, l0);
        split_bf16(v[2 * k + 1], h1, l1);
        h[k] = pack2(h0, h1);
        l[k] = pack2(l0, l1);
    }
    unsigned char* base = qpack + (size_t)tile * 2 * kTileBytes;
    const uint32_t o = tc::kmajor_offset(row, 8 * c);
    *reinterpret_cast<uint4*>(base + o) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(base + kTileBytes + o) = make_uint4(l[0], l[1], l[2], l[3]);
}

// One thread per (group, element) of the packed records.
__global__ void k_pack_tc(int P, int n_neu, const float* __restrict__ W1t, const float* __restrict__ b1t,
                          const float* __restrict__ w2t, const float* __restrict__ b2t,
                          unsigned char* __restrict__ packed)
{
    const int groups = (P + kTcGroup - 1) / kTcGroup;
    const int per = kTile * 32 + kTcGroup * 32 * 32 + kTcGroup * 32;  // w1 elems, w1t elems, bias rows
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= groups * per) return;
    const int g = e / per, r = e % per, k0 = g * kTcGroup;
    const int mg = min(kTcGroup, P - k0);
    unsigned char* rec = packed + (size_t)g * kGroupBytes;
    if (r < kTile * 32) {  // GEMM-1 B row = 32 m + mu, column nu
        const int row = r / 32, nu = r % 32, m = row / 32, mu = row % 32;
        const bool on = m < mg && mu < n_neu;
        put_split(rec, rec + kW1Bytes, row, nu, on ? W1t[((size_t)mu * kNdes + nu) * P + k0 + m] : 0.f);
        return;
    }
    int t = r - kTile * 32;
    if (t < kTcGroup * 32 * 32) {  // GEMM-2 B of member m: row nu, column mu
        const int m = t / 1024, nu = (t / 32) % 32, mu = t % 32;
        const bool on = m < mg && mu < n_neu;
        unsigned char* hi = rec + 2 * kW1Bytes + m * kW1tBytes;
        put_split(hi, hi + kTcGroup * kW1tBytes, nu, mu, on ? W1t[((size_t)mu * kNdes + nu) * P + k0 + m] : 0.f);
        return;
    }
    t -= kTcGroup * 32 * 32;
    float* fb = reinterpret_cast<float*>(rec + 2 * kW1Bytes + 2 * kTcGroup * kW1tBytes);
    const int m = t / 32, mu = t % 32;
    const bool on = m < mg && mu < n_neu;
    fb[m * 32 + mu] = on ? b1t[(size_t)mu * P + k0 + m] : 0.f;
    fb[kTcGroup * 32 + m * 32 + mu] = on ? w2t[(size_t)mu * P + k0 + m] : 0.f;
    if (mu == 0) fb[2 * kTcGroup * 32 + m] = m < mg ? b2t[k0 + m] : 0.f;
}

// Issue the split-BF16 products of one K = 32 tile pair into d_tmem:
// a_hi b_hi + a_hi b_lo (+ a_lo b_hi when a_lo is given).
__device__ __forceinline__ void mma_split(uint32_t d_tmem, const unsigned char* a_hi, const unsigned char* a_lo,
                                          const unsigned char* b_hi, const unsigned char* b_lo, uint32_t idesc)
{
    const unsigned char* as[3] = {a_hi, a_hi, a_lo};
    const unsigned char* bs[3] = {b_hi, b_lo, b_hi};
    const int np = a_lo ? 3 : 2;
    for (int p = 0; p < np; ++p)
        for (int ks = 0; ks < 2; ++ks)
            tc::mma_bf16(d_tmem, tc::smem_desc(tc::smem_u32(as[p]) + ks * 256, 128, 512),
                         tc::smem_desc(tc::smem_u32(bs[p]) + ks * 256, 128, 512), idesc, p > 0 || ks > 0);
}

// Barrier that also orders tcgen05 work and async-proxy shared-memory reads
// around it.
__device__ __forceinline__ void tc_sync()
{
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

// Grid (member groups of 4, atom tiles of 128), groups fastest so the CTAs
// that fill one tile's G rows run together.  Outputs U [N][P] (FP64) and
// G [N][32][Pst] (member innermost; FP32, or FP16 when GH: the contraction
// then reads half the bytes).  The network's arithmetic is the same either way.  Warp w: TMEM lane quarter w & 3 (its 32 atoms),
// half w >> 2 (members {2h, 2h+1} in epilogue 1, descriptors [16h, 16h+16) in
// epilogue 2).
template <bool GH>
__global__ void __launch_bounds__(kPopThreads) k_pop_tc(int N, int P, int Pst, const unsigned char* __restrict__ qpack,
                                                        const unsigned char* __restrict__ packed,
                                                        void* __restrict__ Gv, double* __restrict__ U, unsigned* err)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    PopSmem& S = *reinterpret_cast<PopSmem*>(smem_raw);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int quarter = warp & 3, half = warp >> 2;
    const int row = quarter * 32 + lane;     // tile row = TMEM lane
    const int i = blockIdx.y * kTile + row;  // atom
    const bool valid = i < N;
    const int gi = blockIdx.x, k0 = gi * kTcGroup;

    // ---- GEMM-1 operands by two bulk async copies: the tile's descriptors as
    // split BF16 (16 KB, packed once per training set) and the group's packed
    // weights (33.8 KB, L2-resident records)
    if (t == 0) {
        tc::mbar_init(&S.mbar_ld, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(&S.mbar_ld)),
                     "r"((uint32_t)(2 * kTileBytes + kGroupBytes))
                     : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         tc::smem_u32(S.a)),
                     "l"(qpack + (size_t)blockIdx.y * 2 * kTileBytes), "r"((uint32_t)(2 * kTileBytes)),
                     "r"(tc::smem_u32(&S.mbar_ld))
                     : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         tc::smem_u32(S.grp)),
                     "l"(packed + (size_t)gi * kGroupBytes), "r"((uint32_t)kGroupBytes), "r"(tc::smem_u32(&S.mbar_ld))
                     : "memory");
    }
    if (t == 0) {
        tc::mbar_init(&S.mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        tc::tmem_alloc(&S.tmem_base, kTmemCols);
        tc::tmem_relinquish();
    }
    tc_sync();
    // the group record has landed (bounded wait; a lost copy latches a timeout)
    const bool ld_ok = __syncthreads_and(tc::mbar_wait(&S.mbar_ld, 0, kMaxPolls)) != 0;
    bool ok = ld_ok;
    const uint32_t tb = S.tmem_base;
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    const unsigned char* w1t_hi = S.grp + 2 * kW1Bytes;
    const unsigned char* w1t_lo = w1t_hi + kTcGroup * kW1tBytes;
    const float* fb = reinterpret_cast<const float*>(S.grp + 2 * kW1Bytes + 2 * kTcGroup * kW1tBytes);

    // ---- GEMM 1: H = Q W1^T into TMEM columns [0, 128), member m at [32 m, 32 m + 32)
    if (ok) {
        if (t == 0) {
            mma_split(tb, S.a, S.a + kTileBytes, S.grp, S.grp + kW1Bytes, tc::idesc_bf16_f32(kTile, kTmemCols));
            tc::mma_commit(&S.mbar);
        }
        ok = __syncthreads_and(tc::mbar_wait(&S.mbar, 0, kMaxPolls)) != 0;
    }
    tc::fence_after_sync();
    if (ok) {
        // ---- epilogue 1: x = tanh(H - b1), U, D = w2 (1 - x^2) as BF16 into the GEMM-2 A tiles
#pragma unroll 1
        for (int m = 2 * half; m < 2 * half + 2; ++m) {
            uint32_t r[4][8];
#pragma unroll
            for (int c = 0; c < 4; ++c) tc::tmem_ld8(tb + lane_base + (uint32_t)(32 * m + 8 * c), r[c]);
            tc::tmem_ld_wait();
            float u = 0.f;
            unsigned char* D = d_tile(S, m);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                uint32_t d[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    __nv_bfloat16 dd[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int mu = 8 * c + 2 * e + h;
                        const float x = tanhf(__uint_as_float(r[c][2 * e + h]) - fb[m * 32 + mu]);
                        const float w2 = fb[kTcGroup * 32 + m * 32 + mu];
                        u = fmaf(w2, x, u);
                        dd[h] = __float2bfloat16_rn(w2 * fmaf(-x, x, 1.f));
                    }
                    d[e] = pack2(dd[0], dd[1]);
                }
                *reinterpret_cast<uint4*>(D + tc::kmajor_offset(row, 8 * c)) = make_uint4(d[0], d[1], d[2], d[3]);
            }
            if (valid && k0 + m < P) U[(size_t)i * P + k0 + m] = (double)u - (double)fb[2 * kTcGroup * 32 + m];
        }
    }
    tc_sync();
    // ---- GEMM 2: G_m = D_m W1_m into TMEM columns [32 m, 32 m + 32) (epilogue 1 has read them)
    if (ok) {
        if (t == 0) {
            const uint32_t idesc = tc::idesc_bf16_f32(kTile, 32);
            for (int m = 0; m < kTcGroup; ++m)
                mma_split(tb + 32u * (uint32_t)m, d_tile(S, m), nullptr, w1t_hi + m * kW1tBytes,
                          w1t_lo + m * kW1tBytes, idesc);
            tc::mma_commit(&S.mbar);
        }
        ok = __syncthreads_and(tc::mbar_wait(&S.mbar, 1, kMaxPolls)) != 0;
        tc::fence_after_sync();
    }
    if (ok) {
        // ---- epilogue 2: descriptors [16 half, 16 half + 16) of the atom, 4 members per float4
        uint32_t r[kTcGroup][2][8];
#pragma unroll
        for (int m = 0; m < kTcGroup; ++m)
#pragma unroll
            for (int c = 0; c < 2; ++c) tc::tmem_ld8(tb + lane_base + (uint32_t)(32 * m + 16 * half + 8 * c), r[m][c]);
        tc::tmem_ld_wait();
        if (valid) {
            const size_t o0 = ((size_t)i * kNdes + 16 * half) * Pst + k0;
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const size_t o = o0 + (size_t)(8 * c + e) * Pst;
                    const float g0 = __uint_as_float(r[0][c][e]), g1 = __uint_as_float(r[1][c][e]);
                    const float g2 = __uint_as_float(r[2][c][e]), g3 = __uint_as_float(r[3][c][e]);
                    if (GH) {  // four members as one 8-byte piece (k0 and Pst are multiples of 4)
                        const __half2 a = __floats2half2_rn(g0, g1), b = __floats2half2_rn(g2, g3);
                        uint2 v;
                        v.x = *reinterpret_cast<const uint32_t*>(&a);
                        v.y = *reinterpret_cast<const uint32_t*>(&b);
                        *reinterpret_cast<uint2*>(reinterpret_cast<__half*>(Gv) + o) = v;
                    } else {
                        *reinterpret_cast<float4*>(reinterpret_cast<float*>(Gv) + o) = make_float4(g0, g1, g2, g3);
                    }
                }
        }
    } else if (t == 0) {
        atomicOr(err, kErrTimeout);
    }
    if (!ld_ok) tc::mbar_wait(&S.mbar_ld, 0, kMaxPolls);  // a copy still in flight (bounded)
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tb, kTmemCols);
}

}  // namespace

size_t pop_tc_packed_bytes(int P) { return (size_t)((P + kTcGroup - 1) / kTcGroup) * kGroupBytes; }

int prepare_pop_tc()
{
    int rc = cuda_fail(cudaFuncSetAttribute(k_pop_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)sizeof(PopSmem)), "population kernel shared memory");
    if (rc) return rc;
    return cuda_fail(cudaFuncSetAttribute(k_pop_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)sizeof(PopSmem)), "population kernel shared memory");
}

size_t pop_tc_qpack_bytes(int N) { return (size_t)((N + kTile - 1) / kTile) * 2 * kTileBytes; }

int launch_pack_q_tc(int N, const float* q, unsigned char* qpack, cudaStream_t st)
{
    const int tiles = (N + kTile - 1) / kTile;
    k_pack_q_tc<<<(tiles * kTile * 4 + 255) / 256, 256, 0, st>>>(N, tiles, q, qpack);
    return cuda_fail(cudaGetLastError(), "pack descriptors for the tensor cores");
}

int launch_pop_tc(int N, int P, int Pst, int n_neu, const unsigned char* qpack, const float* W1t, const float* b1t,
                  const float* w2t, const float* b2t, unsigned char* packed, void* G, bool g_half, double* U,
                  unsigned* err, cudaStream_t st)
{
    if (n_neu > 32 || Pst % 4 != 0 || Pst < P) {
        set_error("tensor-core population path needs n_neu <= 32 and a member stride that is a multiple of 4");
        return NEP_ERR_UNSUPPORTED;
    }
    const int groups = (P + kTcGroup - 1) / kTcGroup;
    const int per = kTile * 32 + kTcGroup * 32 * 32 + kTcGroup * 32;
    k_pack_tc<<<(groups * per + 255) / 256, 256, 0, st>>>(P, n_neu, W1t, b1t, w2t, b2t, packed);
    const size_t smem = sizeof(PopSmem);
    auto kern = g_half ? k_pop_tc<true> : k_pop_tc<false>;
    kern<<<dim3(groups, (N + kTile - 1) / kTile), kPopThreads, smem, st>>>(N, P, Pst, qpack, packed, G, U, err);
    return cuda_fail(cudaGetLastError(), "population tensor-core kernel");
}

}  // namespace nep

extern "C" int nep_tc_selftest(const void* A, const void* B, int N, float* D, unsigned* err, void* stream)
{
    if (!A || !B || !D || !err || N < 16 || N > 256 || N % 16 != 0) {
        nep::set_error("nep_tc_selftest: bad arguments (N a multiple of 16 in [16, 256])");
        return NEP_ERR_ARG;
    }
    nep::k_tc_selftest<<<1, 128, 0, (cudaStream_t)stream>>>(static_cast<const __nv_bfloat16*>(A),
                                                            static_cast<const __nv_bfloat16*>(B), N, D, err);
    return nep::cuda_fail(cudaGetLastError(), "tensor-core self-test kernel");
}
