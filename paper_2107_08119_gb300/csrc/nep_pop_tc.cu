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

#include <algorithm>

#include "nep_dataset.cuh"
#include "nep_internal.cuh"
#include "nep_philox.cuh"
#include "nep_recv.cuh"
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
            tc::mma_kind_f16(tb, tc::smem_desc(tc::smem_u32(sA) + ks * 256, 128, 512),
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

// tanh(a) is taken as 1 - 2 / (1 + e^(2a)) with the hardware exponential
// (__expf) and a fast division: absolute error of order 1e-7 for small |a|
// (the subtraction from 1), saturating to +-1 where e^(2a) over- or
// underflows.  The BF16 mode's network only: D = w2 (1 - x^2) is rounded to
// BF16 for GEMM 2 and the losses are held to 1e-3 of the FP32 path, against an
// error of about 1e-6 eV per atom that this gives U.

// Epilogue-1 arithmetic of eight neurons mu = 8c .. 8c + 7 of one (atom,
// member): x = tanh(h - b1) as above, the running sums of w2 x (even and odd
// neurons apart, u2.x and u2.y), and D = w2 (1 - x^2) rounded to BF16, as
// four words of BF16 pairs.  The FP32 arithmetic runs on packed pairs (f32x2:
// two IEEE round-to-nearest results per instruction, the same as two scalar
// operations): h - b1 = fma(b1, -1, h), 1 - q = fma(q, -1, 1), and
// w2 (1 - x^2) as -(w2 (x^2 - 1)) (rounding is symmetric in sign, the sign
// restored on the BF16 bits).  fb14 / fw24: this member's b1 and w2 rows from
// neuron 8c on, as float4.
__device__ __forceinline__ void epi1_eight(const uint32_t (&h)[8], const float4* fb14, const float4* fw24, float2& u2,
                                           uint32_t (&d)[4])
{
    const float2 one2 = make_float2(1.f, 1.f), mone2 = make_float2(-1.f, -1.f), two2 = make_float2(2.f, 2.f);
    const float4 ba = fb14[0], bb = fb14[1], wa = fw24[0], wb = fw24[1];
    const float2 b1p[4] = {make_float2(ba.x, ba.y), make_float2(ba.z, ba.w), make_float2(bb.x, bb.y),
                           make_float2(bb.z, bb.w)};
    const float2 w2p[4] = {make_float2(wa.x, wa.y), make_float2(wa.z, wa.w), make_float2(wb.x, wb.y),
                           make_float2(wb.z, wb.w)};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float2 hv = make_float2(__uint_as_float(h[2 * e]), __uint_as_float(h[2 * e + 1]));
        const float2 a = __ffma2_rn(b1p[e], mone2, hv);  // h - b1
        const float2 t = __fmul2_rn(a, two2);
        const float2 den = __fadd2_rn(one2, make_float2(__expf(t.x), __expf(t.y)));
        const float2 q = make_float2(__fdividef(2.f, den.x), __fdividef(2.f, den.y));
        const float2 x = __ffma2_rn(q, mone2, one2);  // 1 - 2 / (1 + e^(2a))
        u2 = __ffma2_rn(w2p[e], x, u2);
        const float2 dn = __fmul2_rn(w2p[e], __ffma2_rn(x, x, mone2));  // -w2 (1 - x^2)
        const __nv_bfloat162 b = __float22bfloat162_rn(dn);
        d[e] = *reinterpret_cast<const uint32_t*>(&b) ^ 0x80008000u;
    }
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

// One thread per (group, element) of the packed records, read straight from
// the population z [P][n_par] (layout w1 [n_neu][32], b1, w2, b2 per member),
// or (kDraw, an SNES generation) drawn while packing: element e = k n_par + p
// of the generation's normals r (nep_philox.cuh), z = m + s r, each stored by
// the one thread whose record entry owns the element; with draws, the thread
// of a W1 weight's GEMM-1 entry also writes its GEMM-2 entry (the same
// element), and the GEMM-2 range is not launched.
__host__ __device__ constexpr int pack_tc_threads_per_group(bool draw)
{
    return kTile * 32 + (draw ? 0 : kTcGroup * 32 * 32) + kTcGroup * 32;
}

template <bool kDraw>
__global__ void k_pack_tc(int P, int n_neu, const float* __restrict__ z, unsigned char* __restrict__ packed,
                          unsigned long long seed, const unsigned* __restrict__ d_gen, const float* __restrict__ mv,
                          const float* __restrict__ sv, float* __restrict__ r_out, float* __restrict__ z_out)
{
    const int n_par = (kNdes + 2) * n_neu + 1;
    const int groups = (P + kTcGroup - 1) / kTcGroup;
    const int per = pack_tc_threads_per_group(kDraw);  // w1 elems, (w1t elems,) bias rows
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= groups * per) return;
    const unsigned gen = kDraw ? *d_gen : 0u;
    auto val = [&](int k, int p, bool own) -> float {
        const long long el = (long long)k * n_par + p;
        if (!kDraw) return z[el];
        const float g = normal_at(el, gen, seed);
        const float v = fmaf(sv[p], g, mv[p]);
        if (own) {
            r_out[el] = g;
            z_out[el] = v;
        }
        return v;
    };
    const int g = e / per, r = e % per, k0 = g * kTcGroup;
    const int mg = min(kTcGroup, P - k0);
    unsigned char* rec = packed + (size_t)g * kGroupBytes;
    if (r < kTile * 32) {  // GEMM-1 B row = 32 m + mu, column nu
        const int row = r / 32, nu = r % 32, m = row / 32, mu = row % 32;
        const bool on = m < mg && mu < n_neu;
        const float v = on ? val(k0 + m, mu * kNdes + nu, true) : 0.f;
        put_split(rec, rec + kW1Bytes, row, nu, v);
        if (kDraw) {  // GEMM-2 B of member m: row nu, column mu
            unsigned char* hi = rec + 2 * kW1Bytes + m * kW1tBytes;
            put_split(hi, hi + kTcGroup * kW1tBytes, nu, mu, v);
        }
        return;
    }
    int t = r - kTile * 32;
    if (!kDraw && t < kTcGroup * 32 * 32) {  // GEMM-2 B of member m: row nu, column mu
        const int m = t / 1024, nu = (t / 32) % 32, mu = t % 32;
        const bool on = m < mg && mu < n_neu;
        unsigned char* hi = rec + 2 * kW1Bytes + m * kW1tBytes;
        put_split(hi, hi + kTcGroup * kW1tBytes, nu, mu, on ? val(k0 + m, mu * kNdes + nu, false) : 0.f);
        return;
    }
    if (!kDraw) t -= kTcGroup * 32 * 32;
    float* fb = reinterpret_cast<float*>(rec + 2 * kW1Bytes + 2 * kTcGroup * kW1tBytes);
    const int m = t / 32, mu = t % 32;
    const bool on = m < mg && mu < n_neu;
    fb[m * 32 + mu] = on ? val(k0 + m, n_neu * kNdes + mu, true) : 0.f;
    fb[kTcGroup * 32 + m * 32 + mu] = on ? val(k0 + m, n_neu * kNdes + n_neu + mu, true) : 0.f;
    if (mu == 0) fb[2 * kTcGroup * 32 + m] = m < mg ? val(k0 + m, n_neu * (kNdes + 2), true) : 0.f;
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
            tc::mma_kind_f16(d_tmem, tc::smem_desc(tc::smem_u32(as[p]) + ks * 256, 128, 512),
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
// that fill one tile's G rows run together.  Outputs U [N][P] (FP64) and G in
// the layout GL (GLayout: [N][32][Pst] with the members innermost in FP32 or
// FP16, or FP16 per-atom tensor-core tiles for the owner pass; FP16 halves
// the bytes the contraction reads).  The network's arithmetic is the same
// for every layout.  Warp w: TMEM lane quarter w & 3 (its 32 atoms), half
// w >> 2 (members {2h, 2h+1} in epilogue 1, descriptors [16h, 16h+16) in
// epilogue 2).
template <int GL>
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
            float2 u2 = make_float2(0.f, 0.f);
            unsigned char* D = d_tile(S, m);
            // b1 and w2 of the member's 32 neurons: 16-byte broadcast loads
            const float4* b14 = reinterpret_cast<const float4*>(fb + m * 32);
            const float4* w24 = reinterpret_cast<const float4*>(fb + kTcGroup * 32 + m * 32);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                uint32_t d[4];
                epi1_eight(r[c], b14 + 2 * c, w24 + 2 * c, u2, d);
                *reinterpret_cast<uint4*>(D + tc::kmajor_offset(row, 8 * c)) = make_uint4(d[0], d[1], d[2], d[3]);
            }
            const float u = u2.x + u2.y;
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
        if (valid && GL == kGTilesF16) {
            // member k0 + m's descriptors [16 half + 8 c, + 8) are 16 contiguous bytes
            unsigned char* base = reinterpret_cast<unsigned char*>(Gv) + (size_t)i * owner_tc_g_bytes(Pst);
#pragma unroll
            for (int m = 0; m < kTcGroup; ++m)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    uint32_t h[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const __half2 v = __floats2half2_rn(__uint_as_float(r[m][c][2 * e]),
                                                            __uint_as_float(r[m][c][2 * e + 1]));
                        h[e] = *reinterpret_cast<const uint32_t*>(&v);
                    }
                    *reinterpret_cast<uint4*>(base + tc::kmajor_offset(k0 + m, 16 * half + 8 * c)) =
                        make_uint4(h[0], h[1], h[2], h[3]);
                }
        } else if (valid) {
            const size_t o0 = ((size_t)i * kNdes + 16 * half) * Pst + k0;
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const size_t o = o0 + (size_t)(8 * c + e) * Pst;
                    const float g0 = __uint_as_float(r[0][c][e]), g1 = __uint_as_float(r[1][c][e]);
                    const float g2 = __uint_as_float(r[2][c][e]), g3 = __uint_as_float(r[3][c][e]);
                    if (GL == kGRowsF16) {  // four members as one 8-byte piece (k0 and Pst are multiples of 4)
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

// ------------------------------------------------------- pipelined population
// The same network as k_pop_tc, as a persistent kernel with its roles on
// separate warps, so that the copies, both GEMMs and the epilogues of
// successive 128-atom tiles overlap.  One CTA per SM keeps one member group's
// packed record resident and walks its share of the tiles (CTA c: group
// c mod groups, tiles c / groups, c / groups + CTAs per group, ...):
//   warp 16, lane 0  bulk copies: the record once, then each tile's split
//                    BF16 descriptors into one of kPipeQ stages;
//   warp 17, lane 0  the MMAs: GEMM 1 of tile n into TMEM buffer n mod
//                    kPipeT (128 columns each) up to kPipeT - 1 tiles ahead,
//                    GEMM 2 of tile n into the same buffer once its D is in
//                    shared memory (D buffer n mod 2);
//   warps 0-15       the epilogues in the order E1(0) E1(1) E2(0) E1(2)
//                    E2(1) ...: warp w reads TMEM lane quarter w & 3;
//                    epilogue 1 takes member w >> 2 (tanh, U, D as BF16),
//                    epilogue 2 descriptors [8 (w >> 2), + 8) of all four
//                    members (G).
// A TMEM buffer is freed when epilogue 2 of its tile has read it, so with
// four buffers GEMM 1 runs three tiles ahead of the epilogues.  Every value
// is formed by the same operations in the same order as in k_pop_tc, so the
// two kernels give the same bits.  mbarriers order the roles; every wait is
// bounded, and a wait that runs out latches NEP_ERR_TIMEOUT and raises a flag
// on which every role stops; the copy and MMA threads then wait (bounded) for
// their own work in flight before the CTA frees its TMEM.
constexpr int kPipeEpiWarps = 16;
constexpr int kPipeThreads = (kPipeEpiWarps + 2) * 32;
constexpr int kPipeT = 4;  // TMEM buffers of 128 columns (512 columns: one CTA per SM)
constexpr int kPipeQ = 3;  // descriptor stages
constexpr int kPipeD = 2;  // D buffers
struct PipeSmem {
    unsigned char q[kPipeQ][2 * kTileBytes];        // descriptor stages (hi | lo)
    unsigned char d[kPipeD][kTcGroup][kTileBytes];  // D of the four members, per buffer
    unsigned char grp[kGroupBytes];                 // the group's packed record
    uint64_t q_full[kPipeQ], q_empty[kPipeQ], g1_done[kPipeT], g2_done[kPipeT], tmem_free[kPipeT], d_ready[kPipeD];
    uint64_t grp_full, mma_all;
    uint32_t tmem_base;
    int abort;
};

// Bounded wait that also gives up once another role has raised the abort flag.
__device__ __forceinline__ bool pipe_wait(uint64_t* bar, uint32_t parity, volatile int* abort)
{
    const uint32_t a = tc::smem_u32(bar);
    for (uint32_t it = 0; it < kMaxPolls; ++it) {
        uint32_t done = 0;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 31u) == 31u && *abort) return false;
    }
    *abort = 1;
    return false;
}

__device__ __forceinline__ void pipe_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     tc::smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(tc::smem_u32(bar))
                 : "memory");
}

template <int GL>
__global__ void __launch_bounds__(kPipeThreads, 1) k_pop_tc_pipe(int N, int P, int Pst, int groups,
                                                                 const unsigned char* __restrict__ qpack,
                                                                 const unsigned char* __restrict__ packed,
                                                                 void* __restrict__ Gv, double* __restrict__ U,
                                                                 unsigned* err)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    PipeSmem& S = *reinterpret_cast<PipeSmem*>(smem_raw);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int g = blockIdx.x % groups, k0 = g * kTcGroup;
    const int sub = blockIdx.x / groups, nsub = gridDim.x / groups;
    const int tiles = (N + kTile - 1) / kTile;
    const int cnt = sub < tiles ? (tiles - sub + nsub - 1) / nsub : 0;  // this CTA's tiles
    volatile int* abort = &S.abort;
    if (t == 0) {
        for (int b = 0; b < kPipeQ; ++b) {
            tc::mbar_init(&S.q_full[b], 1);
            tc::mbar_init(&S.q_empty[b], 1);
        }
        for (int b = 0; b < kPipeT; ++b) {
            tc::mbar_init(&S.g1_done[b], 1);
            tc::mbar_init(&S.g2_done[b], 1);
            tc::mbar_init(&S.tmem_free[b], kPipeEpiWarps);
        }
        for (int b = 0; b < kPipeD; ++b) tc::mbar_init(&S.d_ready[b], kPipeEpiWarps);
        tc::mbar_init(&S.grp_full, 1);
        tc::mbar_init(&S.mma_all, 1);
        S.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kPipeEpiWarps) {
        tc::tmem_alloc(&S.tmem_base, kPipeT * kTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tb = S.tmem_base;
    const unsigned char* w1t_hi = S.grp + 2 * kW1Bytes;
    const unsigned char* w1t_lo = w1t_hi + kTcGroup * kW1tBytes;
    const float* fb = reinterpret_cast<const float*>(S.grp + 2 * kW1Bytes + 2 * kTcGroup * kW1tBytes);

    if (warp == kPipeEpiWarps) {
        // ---------------------------------------------------------- copies
        if (lane == 0 && cnt > 0) {
            unsigned issued[kPipeQ] = {};
            bulk_copy(S.grp, packed + (size_t)g * kGroupBytes, (uint32_t)kGroupBytes, &S.grp_full);
            for (int n = 0; n < cnt; ++n) {
                const int s = n % kPipeQ, use = n / kPipeQ;
                // the stage's previous tile (n - kPipeQ) has been read by its GEMM 1
                if (use > 0 && !pipe_wait(&S.q_empty[s], (use - 1) & 1, abort)) break;
                bulk_copy(S.q[s], qpack + (size_t)(sub + n * nsub) * 2 * kTileBytes, (uint32_t)(2 * kTileBytes),
                          &S.q_full[s]);
                ++issued[s];
            }
            if (*abort) {  // what is in flight lands before the CTA goes (bounded)
                tc::mbar_wait(&S.grp_full, 0, kMaxPolls);
                for (int s = 0; s < kPipeQ; ++s)
                    if (issued[s]) tc::mbar_wait(&S.q_full[s], (issued[s] - 1) & 1, kMaxPolls);
            }
        }
    } else if (warp == kPipeEpiWarps + 1) {
        // ------------------------------------------------------------ MMAs
        if (lane == 0 && cnt > 0) {
            const uint32_t id1 = tc::idesc_bf16_f32(kTile, kTmemCols), id2 = tc::idesc_bf16_f32(kTile, 32);
            bool ok = pipe_wait(&S.grp_full, 0, abort);
            auto gemm1 = [&](int n) {
                const int s = n % kPipeQ, b = n % kPipeT;
                if (!pipe_wait(&S.q_full[s], (n / kPipeQ) & 1, abort)) return false;
                // TMEM buffer b is free once epilogue 2 of tile n - kPipeT has read it
                if (n >= kPipeT && !pipe_wait(&S.tmem_free[b], (n / kPipeT - 1) & 1, abort)) return false;
                tc::fence_after_sync();
                mma_split(tb + (uint32_t)(b * kTmemCols), S.q[s], S.q[s] + kTileBytes, S.grp, S.grp + kW1Bytes, id1);
                tc::mma_commit(&S.g1_done[b]);
                tc::mma_commit(&S.q_empty[s]);
                return true;
            };
            // GEMM 1 runs kPipeT - 1 tiles ahead: G1(n + kPipeT - 1) waits for
            // epilogue 2 of tile n - 1, which the epilogues reach after
            // epilogue 1 of tile n (the D that G2(n) needs)
            for (int n = 0; ok && n < kPipeT - 1 && n < cnt; ++n) ok = gemm1(n);
            for (int n = 0; ok && n < cnt; ++n) {
                const int b = n % kPipeT, db = n % kPipeD;
                if (!(ok = pipe_wait(&S.d_ready[db], (n / kPipeD) & 1, abort))) break;
                tc::fence_after_sync();
                for (int m = 0; m < kTcGroup; ++m)
                    mma_split(tb + (uint32_t)(b * kTmemCols + 32 * m), S.d[db][m], nullptr, w1t_hi + m * kW1tBytes,
                              w1t_lo + m * kW1tBytes, id2);
                tc::mma_commit(&S.g2_done[b]);
                if (n + kPipeT - 1 < cnt) ok = gemm1(n + kPipeT - 1);
            }
            // every MMA issued has completed before TMEM is freed (bounded)
            tc::mma_commit(&S.mma_all);
            tc::mbar_wait(&S.mma_all, 0, kMaxPolls);
        }
    } else {
        // ------------------------------------------------------- epilogues
        const int quarter = warp & 3, part = warp >> 2;
        const int row = quarter * 32 + lane;
        const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
        bool ok = cnt > 0 && pipe_wait(&S.grp_full, 0, abort);
        // epilogue 1 of tile n: member `part`
        auto epi1 = [&](int n) {
            const int b = n % kPipeT, db = n % kPipeD, m = part;
            if (!pipe_wait(&S.g1_done[b], (n / kPipeT) & 1, abort)) return false;
            tc::fence_after_sync();
            const int i = (sub + n * nsub) * kTile + row;
            uint32_t r[4][8];
#pragma unroll
            for (int c = 0; c < 4; ++c) tc::tmem_ld8(tb + lane_base + (uint32_t)(b * kTmemCols + 32 * m + 8 * c), r[c]);
            tc::tmem_ld_wait();
            float2 u2 = make_float2(0.f, 0.f);
            unsigned char* D = S.d[db][m];
            const float4* b14 = reinterpret_cast<const float4*>(fb + m * 32);
            const float4* w24 = reinterpret_cast<const float4*>(fb + kTcGroup * 32 + m * 32);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                uint32_t d[4];
                epi1_eight(r[c], b14 + 2 * c, w24 + 2 * c, u2, d);
                *reinterpret_cast<uint4*>(D + tc::kmajor_offset(row, 8 * c)) = make_uint4(d[0], d[1], d[2], d[3]);
            }
            const float u = u2.x + u2.y;
            // D is visible to the tensor core, and this warp's TMEM reads are done
            tc::fence_proxy_async_smem();
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) pipe_arrive(&S.d_ready[db]);
            if (i < N && k0 + m < P) U[(size_t)i * P + k0 + m] = (double)u - (double)fb[2 * kTcGroup * 32 + m];
            return true;
        };
        // epilogue 2 of tile n: descriptors [8 part, 8 part + 8) of the four members
        auto epi2 = [&](int n) {
            const int b = n % kPipeT;
            if (!pipe_wait(&S.g2_done[b], (n / kPipeT) & 1, abort)) return false;
            tc::fence_after_sync();
            const int i = (sub + n * nsub) * kTile + row;
            uint32_t r[kTcGroup][8];
#pragma unroll
            for (int m = 0; m < kTcGroup; ++m)
                tc::tmem_ld8(tb + lane_base + (uint32_t)(b * kTmemCols + 32 * m + 8 * part), r[m]);
            tc::tmem_ld_wait();
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) pipe_arrive(&S.tmem_free[b]);
            if (i < N) {
                if (GL == kGTilesF16) {
                    // rows k0..k0+3 of K-chunk `part` are 64 contiguous bytes
                    // (32-byte aligned): two 32-byte stores, whole sectors
                    unsigned char* base = reinterpret_cast<unsigned char*>(Gv) + (size_t)i * owner_tc_g_bytes(Pst);
                    uint32_t h[kTcGroup][4];
#pragma unroll
                    for (int m = 0; m < kTcGroup; ++m)
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const __half2 v = __floats2half2_rn(__uint_as_float(r[m][2 * e]),
                                                                __uint_as_float(r[m][2 * e + 1]));
                            h[m][e] = *reinterpret_cast<const uint32_t*>(&v);
                        }
                    unsigned char* dst = base + tc::kmajor_offset(k0, 8 * part);
#pragma unroll
                    for (int hp = 0; hp < 2; ++hp)
                        asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(dst + 32 * hp),
                                     "r"(h[2 * hp][0]), "r"(h[2 * hp][1]), "r"(h[2 * hp][2]), "r"(h[2 * hp][3]),
                                     "r"(h[2 * hp + 1][0]), "r"(h[2 * hp + 1][1]), "r"(h[2 * hp + 1][2]),
                                     "r"(h[2 * hp + 1][3])
                                     : "memory");
                } else {
                    const size_t o0 = ((size_t)i * kNdes + 8 * part) * Pst + k0;
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const size_t o = o0 + (size_t)e * Pst;
                        const float g0 = __uint_as_float(r[0][e]), g1 = __uint_as_float(r[1][e]);
                        const float g2 = __uint_as_float(r[2][e]), g3 = __uint_as_float(r[3][e]);
                        if (GL == kGRowsF16) {
                            const __half2 a = __floats2half2_rn(g0, g1), c = __floats2half2_rn(g2, g3);
                            uint2 v;
                            v.x = *reinterpret_cast<const uint32_t*>(&a);
                            v.y = *reinterpret_cast<const uint32_t*>(&c);
                            *reinterpret_cast<uint2*>(reinterpret_cast<__half*>(Gv) + o) = v;
                        } else {
                            *reinterpret_cast<float4*>(reinterpret_cast<float*>(Gv) + o) = make_float4(g0, g1, g2, g3);
                        }
                    }
                }
            }
            return true;
        };
        if (ok) ok = epi1(0);
        for (int n = 0; ok && n < cnt; ++n) {
            if (n + 1 < cnt && !(ok = epi1(n + 1))) break;
            ok = epi2(n);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (t == 0 && S.abort) atomicOr(err, kErrTimeout);
    if (warp == kPipeEpiWarps) tc::tmem_dealloc(tb, kPipeT * kTmemCols);
}

// ------------------------------------------------------------ owner pass
// The first contraction pass of the BF16 precision mode on the tensor cores.
// For owner atom j with input gradients G_kj (member k, 32 descriptors) and
// the Jacobians J_q = d q_j / d r of its pairs q, every output of the pass is
// a dot product over the 32 descriptors with G_kj:
//   p_kq^c = sum_d G_kj,d J_q,d^c                       (Eq. 23, partial force)
//   F_kj^c (own term) = sum_d G_kj,d B_j,d^c           (B_j = d q_j / d r_j)
//   W_kj^ab = sum_q -r_q^a p_kq^b = sum_d G_kj,d V_j,d^ab,  V_j^ab = -sum_q r_q^a J_q^b
// so one MMA per tile, D[row][k] = sum_d A[row][d] G[k][d], forms them all
// for every member: A holds a row per (pair, component), own-term component
// and virial component (FP16, packed once per training set), B the owner's G
// tile (FP16, written by the population network), D sits in TMEM.

// J_q,d^c: radial orders d < 8 from the pair record (g_n'/r times r^c), the
// 24 angular descriptors from the pair's angular block (zero beyond r_c^A)
__device__ __forceinline__ float owner_jac(const PairRec& R, long long ai, const float* __restrict__ ang, int d,
                                           int c)
{
    return d < kNR ? R.gd[d] * R.r[c] : (ai >= 0 ? ang[(size_t)ai * (kNA * kLmax * 3) + 3 * (d - kNR) + c] : 0.f);
}

// One block per tile, one thread per row (rows of the padded groups past the
// tile's rows are zero).
__global__ void __launch_bounds__(128) k_pack_owner_tc(const OwnerTile* __restrict__ tiles,
                                                       const PairRec* __restrict__ rec,
                                                       const long long* __restrict__ aidx,
                                                       const float* __restrict__ ang, const float* __restrict__ B,
                                                       const long long* __restrict__ pstart,
                                                       unsigned char* __restrict__ apack, float* __restrict__ rowscale)
{
    const OwnerTile T = tiles[blockIdx.x];
    const int r = threadIdx.x;
    if (r >= 8 * T.groups) return;
    const int np = 3 * T.nt;
    float v[kNdes];
#pragma unroll
    for (int d = 0; d < kNdes; ++d) v[d] = 0.f;
    if (r < np) {
        const long long q = T.q0 + r / 3;
        const int c = r % 3;
        const PairRec R = rec[q];
        const long long ai = aidx[q];
#pragma unroll
        for (int d = 0; d < kNdes; ++d) v[d] = owner_jac(R, ai, ang, d, c);
    } else if (T.extra && r < np + 3) {
        const int c = r - np;
#pragma unroll
        for (int d = 0; d < kNdes; ++d) v[d] = B[((size_t)T.j * kNdes + d) * 3 + c];
    } else if (T.extra && r < np + 9) {
        // xx yy zz xy yz zx
        const int w = r - np - 3, a = w < 3 ? w : w - 3, b = w < 3 ? w : (w - 2) % 3;
        for (long long q = pstart[T.j]; q < pstart[T.j + 1]; ++q) {
            const PairRec R = rec[q];
            const long long ai = aidx[q];
            const float ra = -R.r[a];
#pragma unroll
            for (int d = 0; d < kNdes; ++d) v[d] = fmaf(ra, owner_jac(R, ai, ang, d, b), v[d]);
        }
    }
    // power-of-two row scale: the largest |entry| goes to [2^13, 2^14), far
    // from both ends of the FP16 range; the pass multiplies it back (exactly)
    float mx = 0.f;
#pragma unroll
    for (int d = 0; d < kNdes; ++d) mx = fmaxf(mx, fabsf(v[d]));
    int e = 0;
    if (mx > 0.f) frexpf(mx, &e);  // mx in [2^(e-1), 2^e)
    const int sh = mx > 0.f ? max(-100, min(100, 14 - e)) : 0;
    rowscale[T.row0 + r] = ldexpf(1.f, -sh);
    unsigned char* tile = apack + (size_t)T.row0 * 64;
#pragma unroll
    for (int kc = 0; kc < kNdes / 8; ++kc) {
        uint32_t h[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const __half2 p = __floats2half2_rn(ldexpf(v[8 * kc + 2 * u], sh), ldexpf(v[8 * kc + 2 * u + 1], sh));
            h[u] = *reinterpret_cast<const uint32_t*>(&p);
        }
        *reinterpret_cast<uint4*>(tile + tc::kmajor_offset(r, 8 * kc)) = make_uint4(h[0], h[1], h[2], h[3]);
    }
}

// The owner pass proper: a persistent CTA walks tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ...  Shared memory holds two stages (A tile 8 KB,
// G tile 4 KB), filled by bulk async copies one tile ahead; thread 0 issues
// the copies and the two K = 16 MMAs into 64 TMEM columns; after the MMA has
// completed the four warps read their TMEM lane quarter (thread = tile row)
// into shared memory, and then each warp stores whole rows for members
// 0..Pst-1 (one coalesced store per row): a pair row p_kq^c in FP16 at the
// receiver's slot rev[q], own-term and virial rows in FP32.  Every
// wait is bounded: a timeout latches NEP_ERR_TIMEOUT, the CTA waits (bounded)
// for its copies and MMA still in flight, frees its TMEM and returns.
constexpr int kOtcThreads = 128;
constexpr int kOtcATile = 128 * 64;  // 128 rows x 32 FP16
constexpr int kOtcBTile = 64 * 64;   // up to 64 members x 32 FP16
constexpr int kOtcCols = 64;         // TMEM columns (members)
// epilogue staging of the FP16 pair rows, one half of the member columns at a
// time: 32 halves per row at a stride of 20 words (16-byte row writes by one
// thread each take the minimum four wavefronts), and each row's destination
constexpr int kOtcRowWords = 20;
constexpr int kOtcStageH = 128 * kOtcRowWords * 4;
constexpr int kOtcBars = 64;
constexpr int kOtcSmem = 2 * (kOtcATile + kOtcBTile) + kOtcBars + kOtcStageH + 128 * 8;
constexpr int kOtcPerSm = 6;  // CTAs per SM (35 KB of shared memory and 64 TMEM columns each)

__global__ void __launch_bounds__(kOtcThreads, kOtcPerSm) k_owner_tc(int t0, int t1, const OwnerTile* __restrict__ tiles,
                                                          const unsigned char* __restrict__ apack,
                                                          const float* __restrict__ rowscale,
                                                          const unsigned char* __restrict__ Gt, int Pst,
                                                          const long long* __restrict__ rev, __half* __restrict__ pbuf,
                                                          float* __restrict__ fown, float* __restrict__ w6,
                                                          unsigned* err)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* sA = sm;                       // [2][kOtcATile]
    unsigned char* sB = sm + 2 * kOtcATile;       // [2][kOtcBTile]
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + 2 * (kOtcATile + kOtcBTile));  // [2]
    uint64_t* mbar = full + 2;
    uint32_t* tmem_base = reinterpret_cast<uint32_t*>(mbar + 1);
    uint32_t* stage_h = reinterpret_cast<uint32_t*>(sm + 2 * (kOtcATile + kOtcBTile) + kOtcBars);
    __half** dst = reinterpret_cast<__half**>(stage_h + 128 * kOtcRowWords);
    const int t = threadIdx.x, warp = t >> 5;
    const uint32_t gbytes = (uint32_t)owner_tc_g_bytes(Pst);
    const int nmem = 8 * ((Pst + 7) / 8);          // G rows copied
    const int N = nmem < 16 ? 16 : (nmem + 15) / 16 * 16;  // MMA N (rows past nmem: unused columns)
    const int c8 = (Pst + 7) / 8;                  // 8-column TMEM loads per row
    if (t == 0) {
        tc::mbar_init(&full[0], 1);
        tc::mbar_init(&full[1], 1);
        tc::mbar_init(mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        tc::tmem_alloc(tmem_base, kOtcCols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tb = *tmem_base;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    // copies issued / completions waited per stage, MMAs issued / waited
    unsigned issued[2] = {0u, 0u}, waited[2] = {0u, 0u}, mma_issued = 0u, mma_waited = 0u;
    auto issue = [&](int tile, int s) {
        if (t == 0) {
            const OwnerTile T = tiles[tile];
            const uint32_t abytes = (uint32_t)T.groups * 512u;
            const uint32_t bar = tc::smem_u32(&full[s]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(abytes + gbytes)
                         : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    tc::smem_u32(sA + s * kOtcATile)),
                "l"(apack + (size_t)T.row0 * 64), "r"(abytes), "r"(bar)
                : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    tc::smem_u32(sB + s * kOtcBTile)),
                "l"(Gt + (size_t)T.j * gbytes), "r"(gbytes), "r"(bar)
                : "memory");
        }
        ++issued[s];
    };
    bool ok = true;
    int tile = t0 + (int)blockIdx.x;
    OwnerTile Tn;  // the next tile's record, loaded one tile ahead
    if (tile < t1) {
        issue(tile, 0);
        Tn = tiles[tile];
    }
    for (int it = 0; tile < t1; ++it, tile += (int)gridDim.x) {
        const int s = it & 1;
        const OwnerTile T = Tn;
        if (tile + (int)gridDim.x < t1) Tn = tiles[tile + (int)gridDim.x];
        // this tile's row scales and destinations, loaded before the waits
        const int np = 3 * T.nt, rows = np + (T.extra ? 9 : 0);
        const float sc = t < rows ? rowscale[T.row0 + t] : 0.f;
        const long long rq = t < np ? rev[T.q0 + t / 3] : 0;
        ok = __syncthreads_and(tc::mbar_wait(&full[s], waited[s] & 1u, kMaxPolls)) != 0;
        if (!ok) break;
        ++waited[s];
        tc::fence_after_sync();
        if (t == 0) {
            const uint32_t idesc = tc::idesc_f16_f32(128, N);
            const uint32_t a = tc::smem_u32(sA + s * kOtcATile), b = tc::smem_u32(sB + s * kOtcBTile);
            for (int ks = 0; ks < 2; ++ks)
                tc::mma_kind_f16(tb, tc::smem_desc(a + ks * 256, 128, 512), tc::smem_desc(b + ks * 256, 128, 512),
                                 idesc, ks > 0);
            tc::mma_commit(mbar);
        }
        ++mma_issued;
        // the other stage's previous tile has been consumed by its MMA (waited
        // in the previous iteration): refill it with the next tile
        if (tile + (int)gridDim.x < t1) issue(tile + (int)gridDim.x, s ^ 1);
        ok = __syncthreads_and(tc::mbar_wait(mbar, mma_waited & 1u, kMaxPolls)) != 0;
        if (!ok) break;
        ++mma_waited;
        tc::fence_after_sync();
        // ---- epilogue, in two halves of the member columns (32 each; the
        // second only when Pst > 32), so that a thread holds 32 TMEM values
        // and the staging takes half the shared memory.  1: thread t takes
        // tile row t (TMEM lane t): a pair row half to shared memory as FP16,
        // an own-term or virial row half straight to its FP32 destination
        // (columns past Pst are staged but never stored)
        if (t < np) dst[t] = pbuf + ((size_t)rq * 3 + t % 3) * Pst;
        const int halves = c8 > 4 ? 2 : 1;
        for (int hh = 0; hh < halves; ++hh) {
            uint32_t d[4][8];
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (4 * hh + c < c8) tc::tmem_ld8(tb + lane_base + (uint32_t)(8 * (4 * hh + c)), d[c]);
            tc::tmem_ld_wait();
            if (t < np) {
                uint4* row = reinterpret_cast<uint4*>(stage_h + t * kOtcRowWords);
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (4 * hh + c < c8) {
                        uint32_t h[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const __half2 v = __floats2half2_rn(__uint_as_float(d[c][2 * u]) * sc,
                                                                __uint_as_float(d[c][2 * u + 1]) * sc);
                            h[u] = *reinterpret_cast<const uint32_t*>(&v);
                        }
                        row[c] = make_uint4(h[0], h[1], h[2], h[3]);
                    }
            } else if (t < rows) {
                const int e = t - np;
                float* o = e < 3 ? fown + ((size_t)T.j * 3 + e) * Pst : w6 + ((size_t)T.j * 6 + (e - 3)) * Pst;
#pragma unroll
                for (int c = 0; c < 4; ++c)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int m0 = 8 * (4 * hh + c) + 4 * h;
                        if (m0 < Pst)  // Pst is a multiple of 4
                            *reinterpret_cast<float4*>(o + m0) =
                                make_float4(__uint_as_float(d[c][4 * h]) * sc, __uint_as_float(d[c][4 * h + 1]) * sc,
                                            __uint_as_float(d[c][4 * h + 2]) * sc,
                                            __uint_as_float(d[c][4 * h + 3]) * sc);
                    }
            }
            // this half's TMEM reads are done (the last half's before the next MMA)
            tc::fence_before_sync();
            __syncthreads();
            // ---- 2: the pair row halves, four per warp step: quarter-warp q
            // stores row r + q's half as 8 pieces of 8 bytes (64 contiguous bytes)
            {
                const int lane = t & 31, q = lane >> 3, piece = lane & 7;
                for (int r = 4 * warp + q; r - q < np; r += 4 * (kOtcThreads / 32))
                    if (r < np && 4 * (8 * hh + piece) < Pst)
                        reinterpret_cast<uint2*>(dst[r])[8 * hh + piece] =
                            reinterpret_cast<const uint2*>(stage_h + r * kOtcRowWords)[piece];
            }
            __syncthreads();  // the staging is read before the next half or tile writes it
        }
    }
    if (!ok) {
        if (t == 0) atomicOr(err, kErrTimeout);
        // what is still in flight lands before the TMEM and the CTA go (bounded)
        if (mma_issued > mma_waited) tc::mbar_wait(mbar, mma_waited & 1u, kMaxPolls);
        for (int s = 0; s < 2; ++s)
            if (issued[s] > waited[s]) tc::mbar_wait(&full[s], waited[s] & 1u, kMaxPolls);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tb, kOtcCols);
}
}  // namespace

size_t pop_tc_packed_bytes(int P) { return (size_t)((P + kTcGroup - 1) / kTcGroup) * kGroupBytes; }

int prepare_pop_tc()
{
    int rc = cuda_fail(cudaFuncSetAttribute(k_pop_tc<kGRowsF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)sizeof(PopSmem)), "population kernel shared memory");
    if (!rc)
        rc = cuda_fail(cudaFuncSetAttribute(k_pop_tc<kGRowsF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)sizeof(PopSmem)), "population kernel shared memory");
    if (!rc)
        rc = cuda_fail(cudaFuncSetAttribute(k_pop_tc<kGTilesF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)sizeof(PopSmem)), "population kernel shared memory");
    if (!rc)
        rc = cuda_fail(cudaFuncSetAttribute(k_pop_tc_pipe<kGRowsF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)sizeof(PipeSmem)), "population kernel shared memory");
    if (!rc)
        rc = cuda_fail(cudaFuncSetAttribute(k_pop_tc_pipe<kGTilesF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)sizeof(PipeSmem)), "population kernel shared memory");
    return rc;
}

size_t pop_tc_qpack_bytes(int N) { return (size_t)((N + kTile - 1) / kTile) * 2 * kTileBytes; }

int launch_pack_q_tc(int N, const float* q, unsigned char* qpack, cudaStream_t st)
{
    const int tiles = (N + kTile - 1) / kTile;
    k_pack_q_tc<<<(tiles * kTile * 4 + 255) / 256, 256, 0, st>>>(N, tiles, q, qpack);
    return cuda_fail(cudaGetLastError(), "pack descriptors for the tensor cores");
}

int launch_pop_tc(int N, int P, int Pst, int n_neu, const unsigned char* qpack, const float* z, unsigned char* packed,
                  void* G, int g_layout, double* U, unsigned* err, bool pipelined, cudaStream_t st)
{
    if (n_neu > 32 || Pst % 4 != 0 || Pst < P) {
        set_error("tensor-core population path needs n_neu <= 32 and a member stride that is a multiple of 4");
        return NEP_ERR_UNSUPPORTED;
    }
    const int groups = (P + kTcGroup - 1) / kTcGroup;
    if (z) {
        const int per = pack_tc_threads_per_group(false);
        k_pack_tc<false><<<(groups * per + 255) / 256, 256, 0, st>>>(P, n_neu, z, packed, 0ull, nullptr, nullptr,
                                                                     nullptr, nullptr, nullptr);
    }
    const int tiles = (N + kTile - 1) / kTile;
    if (pipelined && g_layout != kGRowsF32) {
        // one CTA per SM, each keeping one member group's record: as many
        // CTAs per group as fit on the SMs, at most one per tile
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const int nsub = std::max(1, std::min(tiles, nsm / groups));
        auto kp = g_layout == kGTilesF16 ? k_pop_tc_pipe<kGTilesF16> : k_pop_tc_pipe<kGRowsF16>;
        kp<<<groups * nsub, kPipeThreads, sizeof(PipeSmem), st>>>(N, P, Pst, groups, qpack, packed, G, U, err);
        return cuda_fail(cudaGetLastError(), "population tensor-core kernel (pipelined)");
    }
    const size_t smem = sizeof(PopSmem);
    auto kern = g_layout == kGTilesF16 ? k_pop_tc<kGTilesF16>
                                       : (g_layout == kGRowsF16 ? k_pop_tc<kGRowsF16> : k_pop_tc<kGRowsF32>);
    kern<<<dim3(groups, tiles), kPopThreads, smem, st>>>(N, P, Pst, qpack, packed, G, U, err);
    return cuda_fail(cudaGetLastError(), "population tensor-core kernel");
}

int launch_pack_tc_draw(int P, int n_neu, unsigned long long seed, const unsigned* d_gen, const float* m,
                        const float* s, float* r, float* z, unsigned char* packed, cudaStream_t st)
{
    if (n_neu > 32) {
        set_error("tensor-core population path needs n_neu <= 32");
        return NEP_ERR_UNSUPPORTED;
    }
    const int groups = (P + kTcGroup - 1) / kTcGroup;
    const int per = pack_tc_threads_per_group(true);
    k_pack_tc<true><<<(groups * per + 255) / 256, 256, 0, st>>>(P, n_neu, nullptr, packed, seed, d_gen, m, s, r, z);
    return cuda_fail(cudaGetLastError(), "draw and pack the population");
}

int launch_pack_owner_tc(int n_tiles, const OwnerTile* tiles, const PairRec* rec, const long long* aidx,
                         const float* ang, const float* B, const long long* pstart, unsigned char* apack,
                         float* rowscale, cudaStream_t st)
{
    if (n_tiles > 0)
        k_pack_owner_tc<<<n_tiles, 128, 0, st>>>(tiles, rec, aidx, ang, B, pstart, apack, rowscale);
    return cuda_fail(cudaGetLastError(), "pack owner-pass tiles");
}

int prepare_owner_tc()
{
    // kOtcPerSm CTAs per SM need nearly all of the SM's shared memory: ask
    // for the largest carveout
    int rc = cuda_fail(cudaFuncSetAttribute(k_owner_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kOtcSmem),
                       "owner-pass shared memory");
    if (rc) return rc;
    return cuda_fail(cudaFuncSetAttribute(k_owner_tc, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          (int)cudaSharedmemCarveoutMaxShared),
                     "owner-pass shared-memory carveout");
}

int launch_owner_tc(int t0, int t1, const OwnerTile* tiles, const unsigned char* apack, const float* rowscale,
                    const void* G, int Pst, const long long* rev, void* pbuf, float* fown, float* w6, unsigned* err,
                    cudaStream_t st)
{
    if (Pst < 4 || Pst > kOtcCols || Pst % 4 != 0) {
        set_error("tensor-core owner pass: member stride %d outside 4..%d or not a multiple of 4", Pst, kOtcCols);
        return NEP_ERR_UNSUPPORTED;
    }
    if (t1 <= t0) return NEP_OK;
    const int grid = std::min(t1 - t0, 152 * kOtcPerSm);  // persistent: kOtcPerSm CTAs per SM
    k_owner_tc<<<grid, kOtcThreads, kOtcSmem, st>>>(t0, t1, tiles, apack, rowscale,
                                                    static_cast<const unsigned char*>(G), Pst, rev,
                                                    static_cast<__half*>(pbuf), fown, w6, err);
    return cuda_fail(cudaGetLastError(), "tensor-core owner pass");
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
