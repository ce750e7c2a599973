// nep_train.cu -- SNES population evaluation on a training set (Sec. II.D).
//
// Training set: structures of uneven size concatenated into one set of atoms
// (the paper's "super-structure", Sec. II.E), each with its own orthorhombic
// periodic box.  nep_dataset_create precomputes everything that does not
// depend on the parameters z (once):
//   q_i             descriptors [N][32]
//   J_ij            per pair, the derivatives of atom i's descriptor with
//                   respect to r_ij (Eqs. 24-25), stored at i's own slot for
//                   j: radial part as g_n'(r)/r times the vector r_ij (8
//                   floats + vector), angular part 24 x 3
//   B_i             sum over i's own pairs of J_ij ([N][32][3])
// Per population member k the loss then needs only
//   U_ki, G_ki = dU/dq  (network, Eqs. 21-22)
//   p_kji = G_kj . J_ji = dU_kj / dr_ji                           (Eq. 23)
//   F_ki = G_ki . B_i - sum_j p_kji                                (Eqs. 4-5)
//   W_k  = sum_i sum_j r_ij (x) p_kji                              (Eq. 6)
// and the RMSEs of Eqs. 29-34.  Kernels per evaluation:
//   k_pack      z_pop -> member-innermost weight layout (FP32 network; the
//               tensor-core records are packed from z_pop by k_pack_tc)
//   k_mlp_f32   FP32 network per (atom pair, member): U [N][P] and
//               G [N][32][Pst] (member innermost, Pst = P rounded up to 4)
//   k_pop_tc    the same network as BF16 tensor-core GEMMs (nep_pop_tc.cu)
//   k_contract_owner  warp per atom j, two members per lane: p_kji for j's
//               pairs from G_j held in registers, stored at the reverse slot
//   k_contract  warp per atom i: F_i from its slots' p_kji, |F - F_tar|^2,
//               U and W summed per chunk of 32 atoms (k_contract_bulk: the
//               same, the slot rows arriving by bulk copies)
//   k_loss      per member: per-structure sums in a fixed order, RMSEs
// SNES (Eqs. 35-39): k_gauss (Philox4x32-10 normals, z = m + s r; in BF16
// mode the packing kernel draws them itself), k_snes_update.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <new>
#include <type_traits>
#include <vector>

#include <cooperative_groups.h>
#include <cuda_fp16.h>

#include "nep_dataset.cuh"
#include "nep_philox.cuh"
#include "nep_recv.cuh"
#include "nep_tc.cuh"

namespace nep {
namespace {

namespace cg = cooperative_groups;

constexpr int kDsCap = 192;      // neighbour capacity per atom while building (within r_c)
constexpr int kChunkAtoms = 32;       // atoms per contraction block (chunks never span structures)
constexpr int kOwnerMaxThreads = 256;  // owner pass: 4 or 8 warps per block, one atom per warp at a time

inline int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

std::atomic<unsigned long long> g_dataset_uid{0};

// ------------------------------------------------------------------ build
__global__ void k_ds_split(int N, const double* __restrict__ pos, const int* __restrict__ sid,
                           const Box* __restrict__ boxes, const float* __restrict__ zat, float* __restrict__ xh,
                           float* __restrict__ xl, unsigned* __restrict__ err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const Box b = boxes[sid[i]];
    double wx[3];
    for (int d = 0; d < 3; ++d) {
        const double L = b.L[d];
        double x = pos[(size_t)d * N + i];
        if (!isfinite(x)) atomicOr(err, kErrNonFinite);
        double w = x - L * floor(x / L);
        if (w >= L) w -= L;
        if (w < 0.0) w = 0.0;
        wx[d] = w;
    }
    store_pos(xh, xl, i, wx, zat ? zat[i] : 1.f);
}

__global__ void k_ds_list(int N, const int* __restrict__ sid, const int* __restrict__ sstart,
                          const Box* __restrict__ boxes, const float* __restrict__ xh, const float* __restrict__ xl,
                          float rc2, float rcA2, int* __restrict__ tmp, int* __restrict__ cnt, int* __restrict__ cntA,
                          unsigned* err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int s = sid[i];
    const Box b = boxes[s];
    float hi[3], li[3];
    load_pos(xh, xl, N, i, hi, li);
    int c = 0, ca = 0;
    for (int j = sstart[s]; j < sstart[s + 1]; ++j) {
        float hj[3], lj[3];
        load_pos(xh, xl, N, j, hj, lj);
        for (int sx = -b.img[0]; sx <= b.img[0]; ++sx)
            for (int sy = -b.img[1]; sy <= b.img[1]; ++sy)
                for (int sz = -b.img[2]; sz <= b.img[2]; ++sz) {
                    const int code = image_code(sx, sy, sz);
                    if (j == i && code == kImgCenter) continue;
                    float rx, ry, rz;
                    pair_vector(i, j, code, hi, li, hj, lj, b, rx, ry, rz);
                    const float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                    if (d2 < rc2) {
                        if (c < kDsCap) tmp[(size_t)i * kDsCap + c] = j | (code << 24);
                        ++c;
                        if (d2 < rcA2) ++ca;
                    }
                }
    }
    cnt[i] = c;
    cntA[i] = ca;
    if (c > kDsCap) atomicOr(err, kErrOverflow);
}

// Each atom's candidate pairs ordered by increasing distance (ties by the
// search order, so the order is deterministic): the pairs within r_c^A come
// first, so the warps of the fused contraction, whose lanes walk different
// atoms' pairs side by side, run their angular terms together.
__global__ void k_ds_sort(int N, const int* __restrict__ sid, const Box* __restrict__ boxes,
                          const float* __restrict__ xh, const float* __restrict__ xl, const int* __restrict__ cnt,
                          int* __restrict__ tmp)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int c = min(cnt[i], kDsCap);
    const Box b = boxes[sid[i]];
    float hi[3], li[3];
    load_pos(xh, xl, N, i, hi, li);
    int* row = tmp + (size_t)i * kDsCap;
    float key[kDsCap];
    for (int t = 0; t < c; ++t) {
        const int v = row[t];
        const int j = v & 0xFFFFFF;
        float hj[3], lj[3];
        load_pos(xh, xl, N, j, hj, lj);
        float rx, ry, rz;
        pair_vector(i, j, v >> 24, hi, li, hj, lj, b, rx, ry, rz);
        key[t] = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
    }
    // insertion sort (stable): only entries with a strictly larger key move
    for (int t = 1; t < c; ++t) {
        const float kt = key[t];
        const int vt = row[t];
        int u = t - 1;
        while (u >= 0 && key[u] > kt) {
            key[u + 1] = key[u];
            row[u + 1] = row[u];
            --u;
        }
        key[u + 1] = kt;
        row[u + 1] = vt;
    }
}

__global__ void k_ds_compact(int N, const int* __restrict__ tmp, const long long* __restrict__ pstart,
                             const long long* __restrict__ astart, const int* __restrict__ sid,
                             const Box* __restrict__ boxes, const float* __restrict__ xh, const float* __restrict__ xl,
                             float rcA2, int* __restrict__ pj, long long* __restrict__ aidx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const Box b = boxes[sid[i]];
    float hi[3], li[3];
    load_pos(xh, xl, N, i, hi, li);
    const long long p0 = pstart[i], p1 = pstart[i + 1];
    long long a = astart[i];
    for (long long p = p0; p < p1; ++p) {
        const int v = tmp[(size_t)i * kDsCap + (p - p0)];
        pj[p] = v;
        const int j = v & 0xFFFFFF;
        float hj[3], lj[3];
        load_pos(xh, xl, N, j, hj, lj);
        float rx, ry, rz;
        pair_vector(i, j, v >> 24, hi, li, hj, lj, b, rx, ry, rz);
        const float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
        aidx[p] = d2 < rcA2 ? a++ : -1;
    }
}

__global__ void k_ds_reverse(int N, const long long* __restrict__ pstart, const int* __restrict__ pj,
                             long long* __restrict__ rev, unsigned* err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    for (long long p = pstart[i]; p < pstart[i + 1]; ++p) {
        const int v = pj[p];
        const int j = v & 0xFFFFFF;
        const int target = i | ((124 - (v >> 24)) << 24);
        long long found = -1;
        for (long long q = pstart[j]; q < pstart[j + 1]; ++q)
            if (pj[q] == target) {
                found = q;
                break;
            }
        if (found < 0) {
            atomicOr(err, kErrReverse);
            found = p;
        }
        rev[p] = found;
    }
}

// Descriptors of atom i and the Jacobians of its descriptor with respect to
// each of its pair vectors r_ij, scattered to the reverse slots.

__global__ void k_ds_site(int N, const int* __restrict__ sid, const Box* __restrict__ boxes,
                          const float* __restrict__ xh, const float* __restrict__ xl,
                          const long long* __restrict__ pstart, const int* __restrict__ pj,
                          const long long* __restrict__ aidx, float rcR2,
                          float rcA2, float rcR, float rcA, float inv_rcR, float inv_rcA, int typed,
                          float* __restrict__ q_out, float* __restrict__ B_out, PairRec* __restrict__ rec,
                          float* __restrict__ ang)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const Box b = boxes[sid[i]];
    float hi[3], li[3];
    load_pos(xh, xl, N, i, hi, li);
    const float zi = load_z(xh, i);
    float qR[kNR], qC[kNR];
    Harm S;
    for (int a = 0; a < kNR; ++a) qR[a] = qC[a] = 0.f;
    for (int a = 0; a < kNA2; ++a)
        for (int m = 0; m < kLM; ++m) S[a][m] = make_float2(0.f, 0.f);
    const long long p0 = pstart[i], p1 = pstart[i + 1];
    for (long long p = p0; p < p1; ++p) {
        const int v = pj[p];
        const int j = v & 0xFFFFFF;
        float hj[3], lj[3];
        load_pos(xh, xl, N, j, hj, lj);
        float rx, ry, rz;
        pair_vector(i, j, v >> 24, hi, li, hj, lj, b, rx, ry, rz);
        const float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
        const float d = sqrtf(d2);
        const float wz = typed ? sqrtf(zi * load_z(xh, j)) : 1.f;
        if (d2 < rcR2) {
            float g[kNR];
            radial_g<kNR>(d, rcR, inv_rcR, g, wz);
            for (int a = 0; a < kNR; ++a) {
                const float y = g[a] - qC[a];
                const float t = qR[a] + y;
                qC[a] = (t - qR[a]) - y;
                qR[a] = t;
            }
        }
        if (d2 < rcA2) {
            float g[kNA];
            radial_g<kNA>(d, rcA, inv_rcA, g, wz);
            float2 g2[kNA2];
            pair_orders(g, g2);
            float ux, uy, uz;
            unit_vector(rx, ry, rz, ux, uy, uz);
            sh_pass1(ux, uy, uz, g2, S);
        }
    }
    float q[kNdes];
    for (int a = 0; a < kNR; ++a) q[a] = qR[a] - qC[a];
    for (int a = 0; a < kNA; ++a)
        for (int l = 0; l < kLmax; ++l) {
            float s2 = 0.f;
            for (int m = 0; m < kLM; ++m)
                if (sh_l(m) == l) s2 = fmaf(sh_c(m) * harm(S, a, m), harm(S, a, m), s2);
            q[kNR + a * kLmax + l] = s2;
        }
    for (int v = 0; v < kNdes; ++v) q_out[(size_t)i * kNdes + v] = q[v];

    float B[kNdes][3];
    for (int v = 0; v < kNdes; ++v) B[v][0] = B[v][1] = B[v][2] = 0.f;
    for (long long p = p0; p < p1; ++p) {
        const int v = pj[p];
        const int j = v & 0xFFFFFF;
        float hj[3], lj[3];
        load_pos(xh, xl, N, j, hj, lj);
        float r[3];
        pair_vector(i, j, v >> 24, hi, li, hj, lj, b, r[0], r[1], r[2]);
        const float d2 = fmaf(r[0], r[0], fmaf(r[1], r[1], r[2] * r[2]));
        const float d = sqrtf(d2);
        const float inv = 1.f / d;
        const float wz = typed ? sqrtf(zi * load_z(xh, j)) : 1.f;
        PairRec pr;
        pr.r[0] = r[0];
        pr.r[1] = r[1];
        pr.r[2] = r[2];
        pr.pad = 0.f;
        for (int a = 0; a < kNR; ++a) pr.gd[a] = 0.f;
        if (d2 < rcR2) {
            float g[kNR], dg[kNR];
            radial_g_dg<kNR>(d, rcR, inv_rcR, g, dg, wz);
            for (int a = 0; a < kNR; ++a) {
                pr.gd[a] = dg[a] * inv;
                for (int c = 0; c < 3; ++c) B[a][c] = fmaf(pr.gd[a], r[c], B[a][c]);
            }
        }
        rec[p] = pr;  // owner order: the contraction's owner pass streams i's records
        if (d2 < rcA2) {
            float g[kNA], dg[kNA];
            radial_g_dg<kNA>(d, rcA, inv_rcA, g, dg, wz);
            const float u[3] = {r[0] * inv, r[1] * inv, r[2] * inv};
            float Y[kLM], dY[kLM][3];
            sh_eval(u[0], u[1], u[2], Y, dY);
            float J[kNA * kLmax][3];
            for (int t = 0; t < kNA * kLmax; ++t) J[t][0] = J[t][1] = J[t][2] = 0.f;
            for (int m = 0; m < kLM; ++m) {
                const float ud = u[0] * dY[m][0] + u[1] * dY[m][1] + u[2] * dY[m][2];
                float tg[3];
                for (int c = 0; c < 3; ++c) tg[c] = (dY[m][c] - ud * u[c]) * inv;
                const int l = sh_l(m);
                for (int a = 0; a < kNA; ++a) {
                    const float two_s = 2.f * sh_c(m) * harm(S, a, m);
                    for (int c = 0; c < 3; ++c)
                        J[a * kLmax + l][c] = fmaf(two_s, fmaf(dg[a] * Y[m], u[c], g[a] * tg[c]), J[a * kLmax + l][c]);
                }
            }
            const long long ai = aidx[p];
            float* out = ang + (size_t)ai * (kNA * kLmax * 3);
            for (int t = 0; t < kNA * kLmax; ++t)
                for (int c = 0; c < 3; ++c) {
                    out[t * 3 + c] = J[t][c];
                    B[kNR + t][c] += J[t][c];
                }
        }
    }
    for (int v = 0; v < kNdes; ++v)
        for (int c = 0; c < 3; ++c) B_out[((size_t)i * kNdes + v) * 3 + c] = B[v][c];
}

// ------------------------------------------------------------------ evaluation
// z_pop [P][n_par] -> W1t [n_neu][32][P], b1t [n_neu][P], w2t [n_neu][P], b2t [P]
__global__ void k_pack(int P, int n_neu, const float* __restrict__ z, float* __restrict__ W1t,
                       float* __restrict__ b1t, float* __restrict__ w2t, float* __restrict__ b2t)
{
    const int n_par = (kNdes + 2) * n_neu + 1;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P * n_par) return;
    const int k = e / n_par, t = e % n_par;
    const float v = z[e];
    if (t < n_neu * kNdes)
        W1t[(size_t)t * P + k] = v;
    else if (t < n_neu * kNdes + n_neu)
        b1t[(size_t)(t - n_neu * kNdes) * P + k] = v;
    else if (t < n_neu * kNdes + 2 * n_neu)
        w2t[(size_t)(t - n_neu * kNdes - n_neu) * P + k] = v;
    else
        b2t[k] = v;
}

// FP32 network, two atoms per thread (each weight load feeds two FMAs):
// thread t -> atom pair a = t / P, member k = t % P.
__global__ void __launch_bounds__(256) k_mlp_f32(int N, int P, int Pst, int n_neu, const float* __restrict__ q,
                                                 const float* __restrict__ W1t, const float* __restrict__ b1t,
                                                 const float* __restrict__ w2t, const float* __restrict__ b2t,
                                                 float* __restrict__ G, double* __restrict__ U)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long a = t / P;
    const int k = (int)(t % P);
    const long long i0 = 2 * a;
    if (i0 >= N) return;
    const bool two = i0 + 1 < N;
    const long long i1 = two ? i0 + 1 : i0;
    // the two atoms side by side: (atom i0, atom i1) pairs for the f32x2 FMAs
    float2 q2[kNdes], G2[kNdes];
#pragma unroll
    for (int v = 0; v < kNdes; ++v) {
        q2[v] = make_float2(q[i0 * kNdes + v], q[i1 * kNdes + v]);
        G2[v] = make_float2(0.f, 0.f);
    }
    float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;
    for (int mu = 0; mu < n_neu; ++mu) {
        const float* w = W1t + (size_t)mu * kNdes * P + k;
        float2 a = make_float2(0.f, 0.f);
#pragma unroll
        for (int v = 0; v < kNdes; ++v) a = __ffma2_rn(bcast2(w[(size_t)v * P]), q2[v], a);
        const float bb = b1t[(size_t)mu * P + k], ww = w2t[(size_t)mu * P + k];
        const float x0 = tanhf(a.x - bb), x1 = tanhf(a.y - bb);
        float tt, e;
        float p = ww * x0, ep = fmaf(ww, x0, -p);
        two_sum(s0, p, tt, e);
        s0 = tt;
        c0 += e + ep;
        p = ww * x1;
        ep = fmaf(ww, x1, -p);
        two_sum(s1, p, tt, e);
        s1 = tt;
        c1 += e + ep;
        const float2 d = make_float2(ww * fmaf(-x0, x0, 1.f), ww * fmaf(-x1, x1, 1.f));
#pragma unroll
        for (int v = 0; v < kNdes; ++v) G2[v] = __ffma2_rn(d, bcast2(w[(size_t)v * P]), G2[v]);
    }
    const double b2 = (double)b2t[k];
    U[i0 * P + k] = (double)s0 + (double)c0 - b2;
#pragma unroll
    for (int v = 0; v < kNdes; ++v) G[(i0 * kNdes + v) * Pst + k] = G2[v].x;
    if (two) {
        U[i1 * P + k] = (double)s1 + (double)c1 - b2;
#pragma unroll
        for (int v = 0; v < kNdes; ++v) G[(i1 * kNdes + v) * Pst + k] = G2[v].y;
    }
}

// Contraction, pass 1 (owner side): one warp per atom j, lane l holding
// members 2l and 2l + 1.  The lane loads its members' G_j once (registers).
// j's Jacobian records are contiguous (owner order), so the warp stages them
// into shared memory 32 pairs at a time with 16-byte asynchronous copies
// (cp.async, requested before G_j is loaded and the own term formed, so the
// latencies overlap), and then forms p_kji = G_kj . J_ji pair by pair from
// shared memory (broadcast reads), storing it at the slot of the reverse pair
// (i -> j) so that pass 2 finds the partial forces acting on i in i's own
// slot order.  The owner's virial contribution sum_i r_ij (x) p_kji
// (r_ij = -r_ji) goes to W6[j][w][k].  No atomics: every value has one writer.
// A launch covers the owners j0 <= j < j1 (a range of whole structures).
// Element type of the partial-force buffer: FP32, or FP16 in the BF16
// precision mode (half the DRAM traffic of the two passes; each loss term
// averages the per-term rounding over all force components).  Two members
// are stored and loaded together.
__device__ __forceinline__ void pb_store2(float* o, float2 v) { *reinterpret_cast<float2*>(o) = v; }
__device__ __forceinline__ void pb_store2(__half* o, float2 v)
{
    *reinterpret_cast<__half2*>(o) = __floats2half2_rn(v.x, v.y);
}

constexpr int kOwnerChunk = 32;                                     // pairs staged per round
constexpr int kRecFloats = (int)(sizeof(PairRec) / sizeof(float));  // 12
constexpr int kAngFloats = kNA * kLmax * 3;                         // 72
constexpr int kOwnerStage = kOwnerChunk * (kRecFloats + kAngFloats);  // floats per warp

template <class PT>
__global__ void __launch_bounds__(kOwnerMaxThreads) k_contract_owner(
    int j0, int j1, int P, int Pst, const PT* __restrict__ G, const float* __restrict__ B,
    const long long* __restrict__ pstart, const long long* __restrict__ rev, const PairRec* __restrict__ rec,
    const long long* __restrict__ aidx, const float* __restrict__ ang, PT* __restrict__ pbuf,
    float* __restrict__ w6out, float* __restrict__ fown)
{
    extern __shared__ float4 s_stage4[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* s_rec = reinterpret_cast<float*>(s_stage4) + (size_t)warp * kOwnerStage;
    float* s_ang = s_rec + kOwnerChunk * kRecFloats;
    const int k0 = 2 * lane;
    const bool ld = k0 < Pst;  // Pst is even: the float2 at k0 is inside the row
    const int warps = (int)((gridDim.x * blockDim.x) >> 5);
    // 16-byte asynchronous copies global -> shared (no register staging)
    auto cp16 = [](float* dst, const float* src) {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                     "l"(src)
                     : "memory");
    };
    for (int j = j0 + (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); j < j1; j += warps) {
        const long long pe = pstart[j + 1];
        long long q0 = pstart[j];
        int nq = (int)min((long long)kOwnerChunk, pe - q0);
        // the first chunk's pair descriptors and records are requested before
        // G_j and the own term, so their latencies overlap
        long long my_ai = lane < nq ? aidx[q0 + lane] : -1;
        long long my_rv = lane < nq ? rev[q0 + lane] : 0;
        for (int t = lane; t < nq * kRecFloats / 4; t += 32)
            cp16(s_rec + 4 * t, reinterpret_cast<const float*>(rec + q0) + 4 * t);
        float2 g[kNdes];
        const PT* Gj = G + (size_t)j * kNdes * Pst + k0;
#pragma unroll
        for (int v = 0; v < kNdes; ++v) g[v] = ld ? pb_load2(Gj + (size_t)v * Pst) : make_float2(0.f, 0.f);
        // this chunk's angular records are the consecutive ones starting at
        // the first angular pair's index (owner order assigns them in turn)
        unsigned angmask = __ballot_sync(0xffffffffu, my_ai >= 0);
        int na = __popc(angmask);
        long long a0 = na ? __shfl_sync(0xffffffffu, my_ai, __ffs(angmask) - 1) : 0;
        for (int t = lane; t < na * kAngFloats / 4; t += 32)
            cp16(s_ang + 4 * t, ang + (size_t)a0 * kAngFloats + 4 * t);
        asm volatile("cp.async.commit_group;" ::: "memory");
        // own term G_j . B_j (B_j = sum of j's own Jacobians), for pass 2
        {
            const float4* B4 = reinterpret_cast<const float4*>(B + (size_t)j * kNdes * 3);
            float2 f[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
            for (int u = 0; u < kNdes * 3 / 12; ++u) {  // 4 descriptors (12 floats) per step
                const float4 b0 = B4[3 * u], b1 = B4[3 * u + 1], b2 = B4[3 * u + 2];
                const float bb[4][3] = {{b0.x, b0.y, b0.z}, {b0.w, b1.x, b1.y}, {b1.z, b1.w, b2.x},
                                        {b2.y, b2.z, b2.w}};
#pragma unroll
                for (int d = 0; d < 4; ++d)
#pragma unroll
                    for (int c = 0; c < 3; ++c) f[c] = __ffma2_rn(g[4 * u + d], bcast2(bb[d][c]), f[c]);
            }
            if (ld) {
                float* o = fown + (size_t)j * 3 * Pst + k0;
#pragma unroll
                for (int c = 0; c < 3; ++c) *reinterpret_cast<float2*>(o + (size_t)c * Pst) = f[c];
            }
        }
        float2 w6[6];
#pragma unroll
        for (int w = 0; w < 6; ++w) w6[w] = make_float2(0.f, 0.f);
        for (;;) {
            asm volatile("cp.async.wait_all;" ::: "memory");
            __syncwarp();
            for (int t = 0; t < nq; ++t) {
                const float* pr = s_rec + t * kRecFloats;  // r_ji [0..2], g_n'/r [3..10]
                const long long ai = __shfl_sync(0xffffffffu, my_ai, t);
                const long long rq = __shfl_sync(0xffffffffu, my_rv, t);
                // both members of the lane at once (f32x2: two IEEE FMAs per instruction)
                float2 cr = make_float2(0.f, 0.f);
#pragma unroll
                for (int v = 0; v < kNR; ++v) cr = __ffma2_rn(g[v], bcast2(pr[3 + v]), cr);
                const float r0 = pr[0], r1 = pr[1], r2 = pr[2];
                float2 pv[3] = {__fmul2_rn(cr, bcast2(r0)), __fmul2_rn(cr, bcast2(r1)), __fmul2_rn(cr, bcast2(r2))};
                if (ai >= 0) {
                    const float* A = s_ang + (size_t)(ai - a0) * kAngFloats;
#pragma unroll
                    for (int d = 0; d < kNA * kLmax; ++d) {
                        const float2 gg = g[kNR + d];
#pragma unroll
                        for (int c = 0; c < 3; ++c) pv[c] = __ffma2_rn(gg, bcast2(A[3 * d + c]), pv[c]);
                    }
                }
                if (ld) {
                    PT* o = pbuf + (size_t)rq * 3 * Pst + k0;
#pragma unroll
                    for (int c = 0; c < 3; ++c) pb_store2(o + (size_t)c * Pst, pv[c]);
                }
                w6[0] = __ffma2_rn(bcast2(-r0), pv[0], w6[0]);  // xx
                w6[1] = __ffma2_rn(bcast2(-r1), pv[1], w6[1]);  // yy
                w6[2] = __ffma2_rn(bcast2(-r2), pv[2], w6[2]);  // zz
                w6[3] = __ffma2_rn(bcast2(-r0), pv[1], w6[3]);  // xy
                w6[4] = __ffma2_rn(bcast2(-r1), pv[2], w6[4]);  // yz
                w6[5] = __ffma2_rn(bcast2(-r2), pv[0], w6[5]);  // zx
            }
            __syncwarp();  // the stage is refilled by the next chunk
            q0 += kOwnerChunk;
            if (q0 >= pe) break;
            nq = (int)min((long long)kOwnerChunk, pe - q0);
            my_ai = lane < nq ? aidx[q0 + lane] : -1;
            my_rv = lane < nq ? rev[q0 + lane] : 0;
            for (int t = lane; t < nq * kRecFloats / 4; t += 32)
                cp16(s_rec + 4 * t, reinterpret_cast<const float*>(rec + q0) + 4 * t);
            angmask = __ballot_sync(0xffffffffu, my_ai >= 0);
            na = __popc(angmask);
            a0 = na ? __shfl_sync(0xffffffffu, my_ai, __ffs(angmask) - 1) : 0;
            for (int t = lane; t < na * kAngFloats / 4; t += 32)
                cp16(s_ang + 4 * t, ang + (size_t)a0 * kAngFloats + 4 * t);
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        if (ld) {
            float* o = w6out + (size_t)j * 6 * Pst + k0;
#pragma unroll
            for (int w = 0; w < 6; ++w) *reinterpret_cast<float2*>(o + (size_t)w * Pst) = w6[w];
        }
    }
}

// Contraction, pass 2 (receiver side): one block (8 warps) per chunk of <=
// kChunkAtoms atoms of one structure; each warp takes every 8th atom i, lane l
// members 2l and 2l + 1: F_i = G_i . B_i (from pass 1) - sum over i's slots of
// the stored p_kji (coalesced float2 rows, in slot order, UNROLL slots in
// flight).  The per-atom operands (own term, virial terms, U, F_tar, slot
// range) of the warp's next atom are loaded while the current atom's slots
// stream in.  Per chunk and member: sums of U, of |F - F_tar|^2 and of the six
// virial components, in a fixed order (atoms in order within a warp, then the
// warps in order).  A launch covers the chunks c0 <= c < c0 + gridDim.x.
// With `discard` set, a warp that has read an atom's slots drops the 128-byte
// L2 lines lying wholly inside them (discard.global.L2: no write-back of data
// that is dead until the next evaluation rewrites every slot); lines shared
// with a neighbouring atom's slots are left alone.
template <int UNROLL, class PT>
__global__ void __launch_bounds__(kReceiverThreads, 2) k_contract(
    int c0, int discard, int P, int Pst, const int* __restrict__ chunk_begin, const int* __restrict__ chunk_end,
    const double* __restrict__ U, const long long* __restrict__ pstart, const float* __restrict__ fown,
    const PT* __restrict__ pbuf, const float* __restrict__ w6in, const float* __restrict__ f_tar,
    double* __restrict__ partials)
{
    constexpr int kWarps = kReceiverThreads / 32;
    __shared__ RecvRed<kWarps> red;
    const int c = c0 + (int)(gridDim.x - 1 - blockIdx.x);  // last chunk first (as k_contract_bulk)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k0 = 2 * lane;
    const bool on0 = k0 < P, on1 = k0 + 1 < P;
    const bool ld = k0 < Pst;
    // per-lane running sums live in shared memory (this lane's slots only)
    RecvAcc acc;
    const int end = chunk_end[c];
    int i = chunk_begin[c] + warp;
    RecvAtom cur, nxt;
    if (i < end) recv_load(cur, i, P, Pst, k0, ld, on0, on1, U, pstart, fown, w6in, f_tar);
    for (; i < end; i += kWarps) {
        if (i + kWarps < end) recv_load(nxt, i + kWarps, P, Pst, k0, ld, on0, on1, U, pstart, fown, w6in, f_tar);
        float F[2][3] = {{cur.fo[0].x, cur.fo[1].x, cur.fo[2].x}, {cur.fo[0].y, cur.fo[1].y, cur.fo[2].y}};
        if (ld) {
#pragma unroll UNROLL
            for (long long p = cur.ps; p < cur.pe; ++p) {
                const PT* o = pbuf + (size_t)p * 3 * Pst + k0;
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) {
                    const float2 x = pb_load2(o + (size_t)cc * Pst);
                    F[0][cc] -= x.x;
                    F[1][cc] -= x.y;
                }
            }
        }
        if (discard) {  // after every lane's loads of i's slots (the barrier orders them)
            __syncwarp();
            discard_l2_lines(pbuf + (size_t)cur.ps * 3 * Pst, pbuf + (size_t)cur.pe * 3 * Pst, lane);
        }
        acc.add(cur, F);
        cur = nxt;
    }
    acc.store(red.u[warp], red.f[warp], k0);
    __syncthreads();
    recv_chunk_store(red, P, partials + (size_t)c * P * 8);
}

// The receiver pass with the slot rows staged in shared memory: per round a
// warp requests up to kRecvStage slots of its atom (3 rows each) with 8-byte
// asynchronous copies (cp.async, no registers held), waits, and sums them in
// slot order: the same arithmetic as k_contract, twice the bytes in flight.
constexpr int kRecvStage = 16;

template <class PT>
__global__ void __launch_bounds__(kReceiverThreads, 2) k_contract_staged(
    int c0, int discard, int P, int Pst, const int* __restrict__ chunk_begin, const int* __restrict__ chunk_end,
    const double* __restrict__ U, const long long* __restrict__ pstart, const float* __restrict__ fown,
    const PT* __restrict__ pbuf, const float* __restrict__ w6in, const float* __restrict__ f_tar,
    double* __restrict__ partials)
{
    constexpr int kWarps = kReceiverThreads / 32;
    constexpr int kPair = 2 * (int)sizeof(PT);  // bytes of one lane's two members
    __shared__ RecvRed<kWarps> red;
    extern __shared__ __align__(16) unsigned char s_slots_raw[];  // [warps][kRecvStage][3][Pst / 2] member pairs
    const int c = c0 + (int)(gridDim.x - 1 - blockIdx.x);  // last chunk first (as k_contract_bulk)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k0 = 2 * lane;
    const bool on0 = k0 < P, on1 = k0 + 1 < P;
    const bool ld = k0 < Pst;
    const int half = Pst / 2;  // member pairs per row
    unsigned char* stage = s_slots_raw + (size_t)warp * kRecvStage * 3 * half * kPair;
    RecvAcc acc;
    const int end = chunk_end[c];
    int i = chunk_begin[c] + warp;
    RecvAtom cur, nxt;
    if (i < end) recv_load(cur, i, P, Pst, k0, ld, on0, on1, U, pstart, fown, w6in, f_tar);
    for (; i < end; i += kWarps) {
        if (i + kWarps < end) recv_load(nxt, i + kWarps, P, Pst, k0, ld, on0, on1, U, pstart, fown, w6in, f_tar);
        float F[2][3] = {{cur.fo[0].x, cur.fo[1].x, cur.fo[2].x}, {cur.fo[0].y, cur.fo[1].y, cur.fo[2].y}};
        for (long long p0 = cur.ps; p0 < cur.pe; p0 += kRecvStage) {
            const int ns = (int)min((long long)kRecvStage, cur.pe - p0);
            if (ld)
                for (int t = 0; t < ns * 3; ++t) {
                    const PT* src = pbuf + (size_t)(p0 * 3 + t) * Pst + k0;
                    const unsigned dst =
                        (unsigned)__cvta_generic_to_shared(stage + ((size_t)t * half + lane) * kPair);
                    if (kPair == 8)
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
                    else
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
                }
            asm volatile("cp.async.commit_group;\n\tcp.async.wait_all;" ::: "memory");
            if (ld)
                for (int t = 0; t < ns; ++t)
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc) {
                        const float2 x =
                            pb_load2(reinterpret_cast<const PT*>(stage + ((size_t)(3 * t + cc) * half + lane) * kPair));
                        F[0][cc] -= x.x;
                        F[1][cc] -= x.y;
                    }
            __syncwarp();  // each lane reads only its own staged words; kept for the reuse order
        }
        if (discard) {
            __syncwarp();
            discard_l2_lines(pbuf + (size_t)cur.ps * 3 * Pst, pbuf + (size_t)cur.pe * 3 * Pst, lane);
        }
        acc.add(cur, F);
        cur = nxt;
    }
    acc.store(red.u[warp], red.f[warp], k0);
    __syncthreads();
    recv_chunk_store(red, P, partials + (size_t)c * P * 8);
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

template <class PT>
__global__ void __launch_bounds__(kReceiverThreads, 2) k_contract_bulk(
    int c0, int discard, int P, int Pst, const int* __restrict__ chunk_begin, const int* __restrict__ chunk_end,
    const double* __restrict__ U, const long long* __restrict__ pstart, const float* __restrict__ fown,
    const PT* __restrict__ pbuf, const float* __restrict__ w6in, const float* __restrict__ f_tar,
    double* __restrict__ partials, unsigned* __restrict__ err)
{
    extern __shared__ __align__(128) unsigned char s_bulk[];
    BulkSmem& S = *reinterpret_cast<BulkSmem*>(s_bulk);
    bulk_init(S);
    BulkWarp bw;
    // the range's chunks from the last: the owner pass wrote the partial
    // forces in owner order, so the last chunks' rows are the ones most
    // likely still in L2
    const int c = c0 + (int)(gridDim.x - 1 - blockIdx.x);
    if (!bulk_receive_chunk<PT>(c, P, Pst, chunk_begin, chunk_end, U, pstart, fown, pbuf, w6in, f_tar, partials, err,
                                discard != 0, S, bw))
        bulk_drain(S, bw);
}

// Fused contraction: one block per (structure s, group of GM members), the
// structure's force terms accumulated in shared memory, so that no partial
// force p_kji ever reaches DRAM.  Lane l of a warp takes owner atom slot
// l / GM and member g GM + l % GM (32 / GM owner atoms per warp, 8 warps per
// block, the structure's owners in turn).  An owner j loads G_kj once into
// registers, adds its own term G_kj . B_j to F_kj and, pair by pair from its
// Jacobian records (owner order, distance-sorted: the angular pairs first),
// forms p_kji = G_kj . J_ji (Eq. 23) and subtracts it from F_ki (Eqs. 4-5);
// the owner's virial terms sum_i r_ij (x) p_kji (Eq. 6) are summed in
// registers.  The force sums are exact: every term is split into a multiple
// of 2^-8 and a remainder on a 2^-32 grid, both added as int32 with shared
// memory atomics, and integer addition does not depend on the order of the
// atomics.  Then, per member, the structure's sums of U_k, |F_k - F_tar|^2
// and the six virial components: each thread its atoms il = t, t + 256, ...
// in order, then one fixed block tree.  Nothing depends on GM: every member
// count per block gives the same bits.  Shared memory: A x GM x 48 bytes
// (A = the structure's atoms).  A term outside +-2^15 eV/A (or not finite)
// latches the non-finite error bit (the int32 sums could otherwise wrap).
constexpr int kFusedThreads = 256;
constexpr float kFxMax = 32768.f;  // 2^15: with at most 193 terms per atom the int32 sums cannot wrap

__device__ __forceinline__ void fx_add(int* hi, int* lo, float p)
{
    const float h = rintf(p * 256.f);           // p = h 2^-8 + r exactly,
    const float r = fmaf(-h, 0.00390625f, p);   // |r| <= 2^-9
    atomicAdd(hi, __float2int_rn(h));
    atomicAdd(lo, __float2int_rn(r * 4294967296.f));
}

size_t fused_smem_bytes(int amax, int gm) { return (size_t)amax * gm * 48; }

__device__ __forceinline__ float g_load(const float* p) { return *p; }
__device__ __forceinline__ float g_load(const __half* p) { return __half2float(*p); }

template <int GM, class GT>
__global__ void __launch_bounds__(kFusedThreads) k_contract_fused(
    int P, int Pst, int n_groups, const int* __restrict__ s_order, const int* __restrict__ sstart,
    const void* __restrict__ Gv, const double* __restrict__ U, const float* __restrict__ B,
    const long long* __restrict__ pstart, const int* __restrict__ pj, const PairRec* __restrict__ rec,
    const long long* __restrict__ astart, const float* __restrict__ ang, const float* __restrict__ f_tar,
    double* __restrict__ partials, unsigned* __restrict__ err)
{
    constexpr int kApw = 32 / GM;  // owner atoms per warp
    const GT* __restrict__ G = reinterpret_cast<const GT*>(Gv);
    constexpr int kWarps = kFusedThreads / 32;
    extern __shared__ int s_fx[];  // Fh [A][3][GM], Fl [A][3][GM] (int32), W6 [A][6][GM] (FP32)
    const int s = s_order[blockIdx.x / n_groups];
    const int g = blockIdx.x % n_groups;
    const int a0 = sstart[s], A = sstart[s + 1] - a0;
    int* Fh = s_fx;
    int* Fl = s_fx + (size_t)A * 3 * GM;
    float* W6 = reinterpret_cast<float*>(s_fx + (size_t)A * 6 * GM);
    for (int t = threadIdx.x; t < A * 12 * GM; t += kFusedThreads) s_fx[t] = 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kl = lane % GM, slot = lane / GM;
    const int k = g * GM + kl;
    const bool on = k < P;
    bool bad = false;
    for (int base = 0; base < A; base += kWarps * kApw) {
        const int jl = base + warp * kApw + slot;
        if (jl >= A) continue;
        const int j = a0 + jl;
        float gv[kNdes];
#pragma unroll
        for (int v = 0; v < kNdes; ++v) gv[v] = on ? g_load(G + ((size_t)j * kNdes + v) * Pst + k) : 0.f;
        {  // own term G_kj . B_j
            const float4* B4 = reinterpret_cast<const float4*>(B + (size_t)j * kNdes * 3);
            float f[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int u = 0; u < kNdes * 3 / 12; ++u) {
                const float4 b0 = B4[3 * u], b1 = B4[3 * u + 1], b2 = B4[3 * u + 2];
                const float bb[4][3] = {{b0.x, b0.y, b0.z}, {b0.w, b1.x, b1.y}, {b1.z, b1.w, b2.x},
                                        {b2.y, b2.z, b2.w}};
#pragma unroll
                for (int d = 0; d < 4; ++d)
#pragma unroll
                    for (int c = 0; c < 3; ++c) f[c] = fmaf(gv[4 * u + d], bb[d][c], f[c]);
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                bad |= !(fabsf(f[c]) < kFxMax);
                if (on) fx_add(Fh + (jl * 3 + c) * GM + kl, Fl + (jl * 3 + c) * GM + kl, f[c]);
            }
        }
        float w6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        // distance-sorted pairs: j's angular pairs are its first ones, and
        // their Jacobian blocks are consecutive from astart[j] (owner order)
        const long long p0 = pstart[j], pe = pstart[j + 1];
        const long long a0j = astart[j];
        const int na = (int)(astart[j + 1] - a0j), np = (int)(pe - p0);
        auto pair_term = [&](int t, bool angular) {
            const long long p = p0 + t;
            const float4* R4 = reinterpret_cast<const float4*>(rec + p);
            const float4 ra = R4[0], rb = R4[1], rcc = R4[2];  // r_ji, g_n'/r for n = 0..7, pad
            const int il = (pj[p] & 0xFFFFFF) - a0;
            const float gd[kNR] = {ra.w, rb.x, rb.y, rb.z, rb.w, rcc.x, rcc.y, rcc.z};
            float cr = 0.f;
#pragma unroll
            for (int v = 0; v < kNR; ++v) cr = fmaf(gv[v], gd[v], cr);
            float pv[3] = {cr * ra.x, cr * ra.y, cr * ra.z};
            if (angular) {
                const float4* A4 = reinterpret_cast<const float4*>(ang + (size_t)(a0j + t) * (kNA * kLmax * 3));
#pragma unroll
                for (int q = 0; q < kNA * kLmax * 3 / 12; ++q) {  // 4 descriptors (12 floats) per step
                    const float4 x0 = A4[3 * q], x1 = A4[3 * q + 1], x2 = A4[3 * q + 2];
                    const float aa[4][3] = {{x0.x, x0.y, x0.z}, {x0.w, x1.x, x1.y}, {x1.z, x1.w, x2.x},
                                            {x2.y, x2.z, x2.w}};
#pragma unroll
                    for (int d = 0; d < 4; ++d)
#pragma unroll
                        for (int c = 0; c < 3; ++c) pv[c] = fmaf(gv[kNR + 4 * q + d], aa[d][c], pv[c]);
                }
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                bad |= !(fabsf(pv[c]) < kFxMax);
                if (on) fx_add(Fh + (il * 3 + c) * GM + kl, Fl + (il * 3 + c) * GM + kl, -pv[c]);
            }
            w6[0] = fmaf(-ra.x, pv[0], w6[0]);  // xx
            w6[1] = fmaf(-ra.y, pv[1], w6[1]);  // yy
            w6[2] = fmaf(-ra.z, pv[2], w6[2]);  // zz
            w6[3] = fmaf(-ra.x, pv[1], w6[3]);  // xy
            w6[4] = fmaf(-ra.y, pv[2], w6[4]);  // yz
            w6[5] = fmaf(-ra.z, pv[0], w6[5]);  // zx
        };
#pragma unroll 2
        for (int t = 0; t < na; ++t) pair_term(t, true);
#pragma unroll 2
        for (int t = na; t < np; ++t) pair_term(t, false);
        if (on)
#pragma unroll
            for (int w = 0; w < 6; ++w) W6[(jl * 6 + w) * GM + kl] = w6[w];
    }
    if (bad) atomicOr(err, kErrNonFinite);
    __syncthreads();
    for (int kk = 0; kk < GM; ++kk) {
        const int kg = g * GM + kk;
        if (kg >= P) break;
        double v[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int il = threadIdx.x; il < A; il += kFusedThreads) {
            const int i = a0 + il;
            v[0] += U[(size_t)i * P + kg];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int o = (il * 3 + c) * GM + kk;
                const double F = (double)Fh[o] * 0.00390625 + (double)Fl[o] * 2.3283064365386963e-10;
                const double d = F - (double)f_tar[(size_t)i * 3 + c];
                v[1] += d * d;
            }
#pragma unroll
            for (int w = 0; w < 6; ++w) v[2 + w] += (double)W6[(il * 6 + w) * GM + kk];
        }
        // the structure's record (U in FP64, the other terms in FP32)
        __shared__ double tot[8];
        block_sum_store<8>(v, tot);
        __syncthreads();
        ChunkRec* out = reinterpret_cast<ChunkRec*>(partials) + (size_t)s * P + kg;
        if (threadIdx.x == 0) out->u = tot[0];
        if (threadIdx.x >= 1 && threadIdx.x < 8) out->fw[threadIdx.x - 1] = (float)tot[threadIdx.x];
        __syncthreads();  // the block sum's shared scratch serves the next member
    }
}

// The fused contraction for GM members per block, reading G in FP16 (gh) or FP32.
typedef void (*FusedKernel)(int, int, int, const int*, const int*, const void*, const double*, const float*,
                            const long long*, const int*, const PairRec*, const long long*, const float*, const float*,
                            double*, unsigned*);
FusedKernel fused_kernel(int gm, bool gh)
{
    if (gm == 4) return gh ? k_contract_fused<4, __half> : k_contract_fused<4, float>;
    if (gm == 8) return gh ? k_contract_fused<8, __half> : k_contract_fused<8, float>;
    return gh ? k_contract_fused<16, __half> : k_contract_fused<16, float>;
}

// kLossSplit blocks per member (grid P x kLossSplit, one thread-block
// cluster per member), block q taking the structures s = q, q + kLossSplit,
// ...: per structure, the chunk records in order (fixed order; with the fused
// contraction, s_chunk0 NULL, the structure's own record): U in FP64, the
// squared force residuals and the virial sums in FP32; then the squared
// per-atom energy error in FP64 and the per-atom virial errors in FP32; with
// its share of the parameters for L1, L2.  Rank 0 of the member's cluster
// adds the blocks' sums in order, read from their shared memory, and forms
// the RMSEs of Eqs. 30-32 and L1, L2 (Eqs. 33-34).  FP64 arithmetic is slow on
// this part: the work is spread over four times as many SMs as members, and
// every term that comes from FP32 values stays in FP32 until the block sums.
constexpr int kLossSplit = 4;     // blocks per member, each over every fourth structure
constexpr int kLossThreads = 64;

// Reciprocals of the loss means' counts: structures S (L_e), force
// components 3N (L_f), virial components 6S (L_v), parameters (L_1, L_2).
struct LossInv {
    double S, F, V, P;
};

inline LossInv loss_inv(int S, int N, int n_par)
{
    return LossInv{1.0 / S, 1.0 / (3.0 * N), 1.0 / (6.0 * S), 1.0 / n_par};
}

// sqrt(x), x >= 0: the FP32 root refined by one Newton step in FP64, y + (x -
// y^2) / (2 y), the step's divisor in FP32 (relative error of order 1e-14; the
// FP64 square root is a long serial sequence on this part).  Outside the FP32
// range (and for 0, infinity or NaN) the library root.
__device__ __forceinline__ double sqrt_refined(double x)
{
    if (!(x > 1e-30 && x < 1e30)) return sqrt(x);
    const float yf = sqrtf((float)x);
    const double y = (double)yf;
    return fma(fma(-y, y, x), (double)(0.5f / yf), y);
}

__global__ void __cluster_dims__(1, kLossSplit, 1) __launch_bounds__(kLossThreads)
    k_loss(int P, int S, int n_par, const int* __restrict__ s_chunk0, const double* __restrict__ s_inv_na,
           const float* __restrict__ s_vtar, const double* __restrict__ partials, const double* __restrict__ e_tar,
           const float* __restrict__ z, double l_e, double l_f, double l_v, double l_1, double l_2, LossInv inv,
           double* __restrict__ loss)
{
    constexpr int kBatch = 4;  // chunks whose loads are issued together (summed in order)
    const int k = blockIdx.x, q = blockIdx.y, nq = gridDim.y;
    const int stride = nq * blockDim.x;
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};  // se, sf, sv, l1, l2
    {
        // this thread's parameters (a few per member): loaded together, summed
        // in order in FP32, one conversion
        constexpr int kZ = 4;
        float a1 = 0.f, a2 = 0.f;
        for (int p0 = q + nq * threadIdx.x; p0 < n_par; p0 += kZ * stride) {
            float zz[kZ];
#pragma unroll
            for (int u = 0; u < kZ; ++u) {
                const int p = p0 + u * stride;
                zz[u] = p < n_par ? z[(size_t)k * n_par + p] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < kZ; ++u) {
                a1 += fabsf(zz[u]);
                a2 = fmaf(zz[u], zz[u], a2);
            }
        }
        acc[3] = (double)a1;
        acc[4] = (double)a2;
    }
    const ChunkRec* rec = reinterpret_cast<const ChunkRec*>(partials);
    double se = 0.0;
    float sf = 0.f, sv = 0.f;
    for (int s = q + nq * threadIdx.x; s < S; s += stride) {
        // the structure's targets and chunk range first (independent loads):
        // 1 / atoms in FP64 for the energy, the virial targets and 1 / atoms
        // in FP32 for the virial
        const double ia = s_inv_na[s];
        const double et = e_tar[s];
        const float4 t0 = reinterpret_cast<const float4*>(s_vtar)[2 * s];
        const float4 t1 = reinterpret_cast<const float4*>(s_vtar)[2 * s + 1];
        const float wt[6] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y};
        const float iaf = t1.z;
        const int c1 = s_chunk0 ? s_chunk0[s + 1] : s + 1;
        double u = 0.0;
        float fw[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        // per-chunk records, or (s_chunk0 NULL) one record per structure: the
        // first 36 bytes of each as three 16-byte loads
        for (int c0 = s_chunk0 ? s_chunk0[s] : s; c0 < c1; c0 += kBatch) {
            uint4 b[kBatch][3];
#pragma unroll
            for (int r = 0; r < kBatch; ++r) {
                const uint4* src = reinterpret_cast<const uint4*>(rec + (size_t)(c0 + r) * P + k);
#pragma unroll
                for (int w = 0; w < 3; ++w) b[r][w] = c0 + r < c1 ? src[w] : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int r = 0; r < kBatch; ++r)
                if (c0 + r < c1) {
                    u += __hiloint2double((int)b[r][0].y, (int)b[r][0].x);
                    const uint32_t f7[7] = {b[r][0].z, b[r][0].w, b[r][1].x, b[r][1].y, b[r][1].z, b[r][1].w,
                                            b[r][2].x};
#pragma unroll
                    for (int w = 0; w < 7; ++w) fw[w] += __uint_as_float(f7[w]);
                }
        }
        const double de = (u - et) * ia;
        se = fma(de, de, se);
        sf += fw[0];
#pragma unroll
        for (int w = 0; w < 6; ++w) {
            const float dv = (fw[1 + w] - wt[w]) * iaf;
            sv = fmaf(dv, dv, sv);
        }
    }
    acc[0] = se;
    acc[1] = (double)sf;
    acc[2] = (double)sv;
    // the block's five sums into its shared memory; rank 0 of the cluster
    // (the member's four blocks) reads the four rows in order and forms the
    // losses; the second cluster barrier keeps every row alive until then
    __shared__ double part[5];
    __shared__ double L[5];
    block_sum_store<5>(acc, part);
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();
    if (cl.block_rank() == 0) {
        // thread c forms term c: the mean over its count (reciprocals from the
        // host: FP64 division is a long serial sequence here), then the root
        if (threadIdx.x < 5) {
            const int c = threadIdx.x;
            double t = 0.0;
            for (int r = 0; r < nq; ++r) t += *cl.map_shared_rank(&part[c], r);
            const double mean = t * (c == 0 ? inv.S : c == 1 ? inv.F : c == 2 ? inv.V : inv.P);
            L[c] = c == 3 ? mean : sqrt_refined(mean);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double* out = loss + (size_t)k * 6;
            out[0] = l_e * L[0] + l_f * L[1] + l_v * L[2] + l_1 * L[3] + l_2 * L[4];
            for (int c = 0; c < 5; ++c) out[1 + c] = L[c];
        }
    }
    cl.sync();
}

// ------------------------------------------------------------------ SNES
// Standard normals for elements e = 0..count-1 of stream (seed, gen): block
// e/4 uses counter {e/4, 0, gen, 0x4E4550} and key {seed lo, seed hi};
// u = (w + 1/2) 2^-32; lanes 0/1 (2/3) are the Box-Muller pair of (u0, u1)
// ((u2, u3)).  Also writes z = m + s (.) r for a population of n_par-vectors.
__global__ void k_gauss(long long count, int n_par, unsigned long long seed, const unsigned* __restrict__ d_gen,
                        const float* __restrict__ m, const float* __restrict__ s, float* __restrict__ r,
                        float* __restrict__ z)
{
    const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (4 * b >= count) return;
    uint32_t w[4];
    philox_block(b, *d_gen, seed, w);
    float g[4];
    box_muller(w[0], w[1], g[0], g[1]);
    box_muller(w[2], w[3], g[2], g[3]);
    for (int l = 0; l < 4; ++l) {
        const long long e = 4 * b + l;
        if (e < count) {
            r[e] = g[l];
            if (z) {
                const int p = (int)(e % n_par);
                z[e] = fmaf(s[p], g[l], m[p]);
            }
        }
    }
}

// z = m + s (.) r for given draws.
__global__ void k_make_pop(long long count, int n_par, const float* __restrict__ m, const float* __restrict__ s,
                           const float* __restrict__ r, float* __restrict__ z)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count) return;
    const int p = (int)(e % n_par);
    z[e] = fmaf(s[p], r[e], m[p]);
}

constexpr int kUpdateThreads = 128;  // parameters per update block (at least kMaxPop)
static_assert(kUpdateThreads >= kMaxPop, "one thread per member in the ranking");

// Where a run of generations keeps its loss history: row (generation - base).
struct SnesCtl {
    double* hist;   // dev [n_gen][P][6] or NULL
    unsigned base;  // generation counter at the start of the run
};

__global__ void k_set_ctl(SnesCtl* ctl, double* hist, unsigned base)
{
    ctl->hist = hist;
    ctl->base = base;
}

// Rank the members by (loss, index), then the natural gradients (Eqs. 36-37)
// with the rank utilities `util` and the update of m with the pre-update s
// (Eq. 38), then s (Eq. 39).  Every block ranks the (few) members itself and
// updates its own slice of parameters; a thread's draws of every member and
// its m and s do not depend on the ranking and are loaded before it, and the
// gradient sums run over the members in index order, each draw weighted by
// the utility of its member's rank.  Block 0 also appends the losses to the
// run's history (ctl, may be NULL) and advances the device generation
// counter that the next generation's draws read.
__global__ void __launch_bounds__(kUpdateThreads) k_snes_update(int P, int n_par, const double* __restrict__ loss,
                                                               const float* __restrict__ util,
                                                               const float* __restrict__ r, float* __restrict__ m,
                                                               float* __restrict__ s, float eta_m, float eta_s,
                                                               int* __restrict__ order_out,
                                                               unsigned* __restrict__ d_gen,
                                                               const SnesCtl* __restrict__ ctl)
{
    __shared__ float ut[kMaxPop];  // utility of rank j
    __shared__ float uk[kMaxPop];  // utility of member k's rank (0 past P)
    __shared__ unsigned long long key[kMaxPop];
    const int t = threadIdx.x;
    const int p = blockIdx.x * blockDim.x + t;
    const bool live = p < n_par;
    float rv[kMaxPop];
#pragma unroll
    for (int k = 0; k < kMaxPop; ++k) rv[k] = live && k < P ? r[(size_t)k * n_par + p] : 0.f;
    const float mp = live ? m[p] : 0.f, sp = live ? s[p] : 0.f;

    // the members' losses as unsigned keys in the same order as the FP64
    // values (integer compares: FP64 compares are slow on this part); -0 is
    // taken as +0, and a NaN loss ranks after every number
    if (t < P) {
        const double l = loss[(size_t)t * 6];
        const long long b = isnan(l) ? 0x7FF8000000000000LL : __double_as_longlong(l + 0.0);
        key[t] = b < 0 ? ~(unsigned long long)b : ((unsigned long long)b | 0x8000000000000000ull);
        ut[t] = util[t];
    }
    __syncthreads();
    if (blockIdx.x == 0) {
        const unsigned g = *d_gen;
        double* hist = ctl ? ctl->hist : nullptr;
        if (hist) {
            double* row = hist + (size_t)(g - ctl->base) * P * 6;
            for (int e = t; e < P * 6; e += blockDim.x) row[e] = loss[e];
        }
        __syncthreads();
        if (t == 0) *d_gen = g + 1;
    }
    if (t < kMaxPop) {
        float w = 0.f;
        if (t < P) {
            const unsigned long long kk = key[t];
            int rank = 0;
            for (int j = 0; j < P; ++j) {
                const unsigned long long kj = key[j];
                rank += (kj < kk || (kj == kk && j < t)) ? 1 : 0;
            }
            w = ut[rank];
            if (order_out && blockIdx.x == 0) order_out[rank] = t;
        }
        uk[t] = w;
    }
    __syncthreads();
    if (!live) return;
    float gm = 0.f, gs = 0.f;
#pragma unroll
    for (int k = 0; k < kMaxPop; ++k) {
        gm = fmaf(uk[k], rv[k], gm);
        gs = fmaf(uk[k], fmaf(rv[k], rv[k], -1.f), gs);
    }
    m[p] = fmaf(eta_m * sp, gm, mp);
    s[p] = sp * expf(0.5f * eta_s * gs);
}

// Deterministic stand-in parameters for timing launch shapes: uniform in
// [-0.1, 0.1] from an integer hash of the element index (Wellons' lowbias32).
__global__ void k_tune_pop(long long count, float* __restrict__ z)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count) return;
    uint32_t x = (uint32_t)e * 2654435761u + 12345u;
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    z[e] = 0.1f * (2.f * ((float)(x >> 8) * (1.f / 16777216.f)) - 1.f);
}

// Largest dynamic shared memory of a fused contraction block (the block sum
// takes 2 KB of static shared memory beside it, out of 227 KB).
constexpr size_t kFusedSmemMax = (size_t)220 * 1024;

bool fused_fits(const nep_dataset* ds, int gm) { return fused_smem_bytes(ds->amax, gm) <= kFusedSmemMax; }

bool valid_shape(const nep_dataset* ds, const EvalShape& h)
{
    return h.waves >= 1 && h.waves <= kMaxWaves && (h.owner_warps == 4 || h.owner_warps == 8) &&
           (h.discard == 0 || h.discard == 1) && (h.mlp_threads == 128 || h.mlp_threads == 256) &&
           (h.recv_unroll == 1 || h.recv_unroll == 4 || h.recv_unroll == 8 || h.recv_unroll == 12 || h.recv_unroll == 16) &&
           (h.fused == 0 || ((h.fused == 4 || h.fused == 8 || h.fused == 16) && fused_fits(ds, h.fused))) &&
           (h.owner_tc == 0 || h.owner_tc == 1) && (h.pop_pipe == 0 || h.pop_pipe == 1);
}

}  // namespace
}  // namespace nep

using namespace nep;


struct snes_state {
    nep_model* m = nullptr;
    int P = 0, n_par = 0;
    unsigned long long seed = 0;
    unsigned gen = 0;
    float* mean = nullptr;
    float* sigma = nullptr;
    float* r = nullptr;
    float* z = nullptr;
    double* loss = nullptr;
    int* order = nullptr;
    float* util = nullptr;  // rank utilities u_1..u_P (a constant of P)
    unsigned* d_gen = nullptr;  // generation counter read by the draws (device)
    nep::SnesCtl* d_ctl = nullptr;
    // one generation captured as a CUDA graph (snes_run), keyed by what it bakes in
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long key_uid = 0;
    int key_epoch = -1, key_prec = -1;
    double key_lam[5] = {0, 0, 0, 0, 0};
};

namespace {

template <class T>
int dalloc(T** p, size_t count, long long* bytes)
{
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        set_error("cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
        return NEP_ERR_OOM;
    }
    if (bytes) *bytes += (long long)(count * sizeof(T));
    return NEP_OK;
}

template <class T>
void dfree(T*& p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

// member stride of G: a multiple of 4 so that a tensor-core member group
// (4 members) is one aligned 16-byte store
inline int member_stride(int P) { return (P + 3) / 4 * 4; }

int ensure_pop(nep_dataset* ds, int P)
{
    if (P <= ds->pop_cap) return NEP_OK;
    dfree(ds->W1t);
    dfree(ds->b1t);
    dfree(ds->w2t);
    dfree(ds->b2t);
    dfree(ds->G);
    dfree(ds->U);
    dfree(ds->partials);
    dfree(ds->packed);
    dfree(ds->pbuf);
    dfree(ds->w6);
    dfree(ds->fown);
    ds->pop_cap = 0;
    const int nn = ds->m->hp.n_neu;
    int rc;
    if ((rc = dalloc(&ds->W1t, (size_t)nn * kNdes * P, nullptr)) || (rc = dalloc(&ds->b1t, (size_t)nn * P, nullptr)) ||
        (rc = dalloc(&ds->w2t, (size_t)nn * P, nullptr)) || (rc = dalloc(&ds->b2t, (size_t)P, nullptr)) ||
        (rc = dalloc(&ds->G, (size_t)ds->N * kNdes * member_stride(P), nullptr)) ||
        (rc = dalloc(&ds->U, (size_t)ds->N * P, nullptr)) ||
        (rc = dalloc(&ds->partials, (size_t)ds->n_chunks * P * 8, nullptr)) ||
        (rc = dalloc(&ds->packed, pop_tc_packed_bytes(P), nullptr)) ||
        (rc = dalloc(&ds->pbuf, (size_t)ds->n_pairs * 3 * member_stride(P), nullptr)) ||
        (rc = dalloc(&ds->w6, (size_t)ds->N * 6 * member_stride(P), nullptr)) ||
        (rc = dalloc(&ds->fown, (size_t)ds->N * 3 * member_stride(P), nullptr)))
        return rc;
    // members past P in the last group of G are never written: keep them zero
    rc = cuda_fail(cudaMemset(ds->G, 0, sizeof(float) * (size_t)ds->N * kNdes * member_stride(P)), "clear G");
    if (rc) return rc;
    ds->pop_cap = P;
    return NEP_OK;
}

// Everything an evaluation with P members needs that must not happen inside a
// stream capture: scratch allocation, kernel attributes, the second stream
// and its events.
int prepare_evaluation(nep_dataset* ds, int P)
{
    const int cap0 = ds->pop_cap;
    int rc = ensure_pop(ds, P);
    if (rc) return rc;
    if (ds->pop_cap != cap0) ++ds->epoch;
    if (!ds->aux) {
        if ((rc = cuda_fail(cudaStreamCreateWithFlags(&ds->aux, cudaStreamNonBlocking), "evaluation stream")))
            return rc;
        for (int w = 0; w < kMaxWaves; ++w)
            if ((rc = cuda_fail(cudaEventCreateWithFlags(&ds->ev_wave[w], cudaEventDisableTiming), "evaluation event")))
                return rc;
        if ((rc = cuda_fail(cudaEventCreateWithFlags(&ds->ev_join, cudaEventDisableTiming), "evaluation event")))
            return rc;
    }
    const int ostage = (kOwnerMaxThreads / 32) * kOwnerStage * (int)sizeof(float);
    const int rstage = (kReceiverThreads / 32) * kRecvStage * 3 * member_stride(kMaxPop) * (int)sizeof(float);
    if ((rc = cuda_fail(cudaFuncSetAttribute(k_contract_owner<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             ostage), "contraction shared memory")) ||
        (rc = cuda_fail(cudaFuncSetAttribute(k_contract_owner<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             ostage), "contraction shared memory")) ||
        (rc = cuda_fail(cudaFuncSetAttribute(k_contract_staged<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             rstage), "contraction shared memory")) ||
        (rc = cuda_fail(cudaFuncSetAttribute(k_contract_staged<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             rstage / 2), "contraction shared memory")) ||
        (rc = cuda_fail(cudaFuncSetAttribute(k_contract_bulk<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(BulkSmem)), "contraction shared memory")) ||
        (rc = cuda_fail(cudaFuncSetAttribute(k_contract_bulk<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(BulkSmem)), "contraction shared memory")))
        return rc;
    for (int gm = 4; gm <= 16; gm *= 2) {
        if (!fused_fits(ds, gm)) continue;
        const int smem = (int)fused_smem_bytes(ds->amax, gm);
        for (int h = 0; h < 2; ++h)
            if ((rc = cuda_fail(cudaFuncSetAttribute(fused_kernel(gm, h != 0),
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                                "fused contraction shared memory")))
                return rc;
    }
    if ((rc = prepare_owner_tc())) return rc;
    return prepare_pop_tc();
}

// The two contraction passes over the chunk range [c_lo, c_hi) (whole
// structures): pass 1 on st, pass 2 on `p2`.
template <class PT>
void launch_contraction_t(const nep_dataset* ds, int P, int Pst, int c_lo, int c_hi, cudaStream_t st,
                          cudaStream_t p2, bool fork, cudaEvent_t ev)
{
    const EvalShape& sh = ds->shape;
    const int ow = sh.owner_warps == 8 ? 8 : 4;
    const int a0 = ds->h_cb[c_lo], a1 = ds->h_ce[c_hi - 1];
    const size_t ostage = (size_t)ow * kOwnerStage * sizeof(float);
    PT* pbuf = reinterpret_cast<PT*>(ds->pbuf);
    if (std::is_same<PT, __half>::value && sh.owner_tc) {
        // the owners' tiles, G in the tensor-core tile layout (a launch error
        // is read back by the caller's cudaGetLastError)
        launch_owner_tc(ds->h_tile0[a0], ds->h_tile0[a1], ds->tiles, ds->apack, ds->rowscale, ds->G, Pst, ds->rev,
                        pbuf, ds->fown, ds->w6, ds->m->d_err, st);
    } else {
        k_contract_owner<PT><<<std::min(blocks_for(a1 - a0, ow), 152 * 64 / ow), 32 * ow, ostage, st>>>(
            a0, a1, P, Pst, reinterpret_cast<const PT*>(ds->G), ds->B, ds->pstart, ds->rev, ds->rec, ds->aidx,
            ds->ang, pbuf, ds->w6, ds->fown);
    }
    if (fork) {
        cudaEventRecord(ev, st);
        cudaStreamWaitEvent(p2, ev, 0);
    }
    if (sh.recv_unroll == 1) {
        k_contract_bulk<PT><<<c_hi - c_lo, kReceiverThreads, sizeof(BulkSmem), p2>>>(
            c_lo, sh.discard, P, Pst, ds->chunk_begin, ds->chunk_end, ds->U, ds->pstart, ds->fown, pbuf, ds->w6,
            ds->f_tar, ds->partials, ds->m->d_err);
    } else if (sh.recv_unroll == 16) {
        const size_t smem = (size_t)(kReceiverThreads / 32) * kRecvStage * 3 * Pst * sizeof(PT);
        k_contract_staged<PT><<<c_hi - c_lo, kReceiverThreads, smem, p2>>>(c_lo, sh.discard, P, Pst, ds->chunk_begin,
                                                                           ds->chunk_end, ds->U, ds->pstart,
                                                                           ds->fown, pbuf, ds->w6, ds->f_tar,
                                                                           ds->partials);
    } else {
        auto recv = sh.recv_unroll == 12 ? k_contract<12, PT> : (sh.recv_unroll == 8 ? k_contract<8, PT> : k_contract<4, PT>);
        recv<<<c_hi - c_lo, kReceiverThreads, 0, p2>>>(c_lo, sh.discard, P, Pst, ds->chunk_begin, ds->chunk_end,
                                                       ds->U, ds->pstart, ds->fown, pbuf, ds->w6, ds->f_tar,
                                                       ds->partials);
    }
}

// The two contraction passes over the chunk range [c_lo, c_hi) (whole
// structures): pass 1 on st, pass 2 on `p2`; the partial forces in FP16 when
// `half` (BF16 precision mode), else FP32.
void launch_contraction(const nep_dataset* ds, int P, int Pst, int c_lo, int c_hi, cudaStream_t st,
                        cudaStream_t p2, bool fork, cudaEvent_t ev, bool half)
{
    if (half)
        launch_contraction_t<__half>(ds, P, Pst, c_lo, c_hi, st, p2, fork, ev);
    else
        launch_contraction_t<float>(ds, P, Pst, c_lo, c_hi, st, p2, fork, ev);
}

// Launches of one population evaluation (no allocation, no attribute calls:
// safe inside a stream capture once prepare_evaluation has run).  With
// shape.waves = W > 1 the contraction runs over up to W consecutive ranges of
// whole structures with about equal pair counts; pass 2 of range w (second
// stream) overlaps pass 1 of range w + 1, and a range's partial forces are
// read back while they are still in L2.  A range never splits a structure:
// pass 1 of a structure's owners writes into the slots of all its atoms.
// prepacked: (BF16) the tensor-core records already hold z_pop (an SNES
// generation that drew and packed in one launch)
int enqueue_evaluation(nep_model* m, nep_dataset* ds, const float* z_pop, int P, int precision,
                       const double* lambdas, double* loss, cudaStream_t st, bool prepacked = false)
{
    if (precision != NEP_PREC_FP32 && precision != NEP_PREC_BF16) {
        set_error("snes_evaluate_population: unknown precision %d", precision);
        return NEP_ERR_ARG;
    }
    const int nn = m->hp.n_neu, n_par = m->n_par, Pst = member_stride(P);
    const EvalShape& sh = ds->shape;
    int rc;
    if (precision == NEP_PREC_BF16) {
        // G in FP16: the contraction reads half the bytes (the loss terms
        // average its rounding over all force components)
        const int layout = !sh.fused && sh.owner_tc ? kGTilesF16 : kGRowsF16;
        if ((rc = launch_pop_tc(ds->N, P, Pst, nn, ds->qpack, prepacked ? nullptr : z_pop, ds->packed, ds->G, layout,
                                ds->U, m->d_err, sh.pop_pipe != 0, st)))
            return rc;
    } else {
        k_pack<<<blocks_for((long long)P * n_par, 256), 256, 0, st>>>(P, nn, z_pop, ds->W1t, ds->b1t, ds->w2t,
                                                                      ds->b2t);
        const long long pairs = (ds->N + 1) / 2;
        const int mt = sh.mlp_threads == 128 ? 128 : 256;
        k_mlp_f32<<<blocks_for(pairs * P, mt), mt, 0, st>>>(ds->N, P, Pst, nn, ds->q, ds->W1t, ds->b1t, ds->w2t,
                                                            ds->b2t, ds->G, ds->U);
    }
    const double lam[5] = {lambdas ? lambdas[0] : 1.0, lambdas ? lambdas[1] : 1.0, lambdas ? lambdas[2] : 1.0,
                           lambdas ? lambdas[3] : 0.05, lambdas ? lambdas[4] : 0.05};
    if (sh.fused) {
        // one block per (structure, member group), largest structures first
        const int gm = sh.fused, groups = (P + gm - 1) / gm;
        const size_t smem = fused_smem_bytes(ds->amax, gm);
        const bool gh = precision == NEP_PREC_BF16;
        fused_kernel(gm, gh)<<<ds->S * groups, kFusedThreads, smem, st>>>(
            P, Pst, groups, ds->s_order, ds->sstart, ds->G, ds->U, ds->B, ds->pstart, ds->pj, ds->rec, ds->astart,
            ds->ang, ds->f_tar, ds->partials, m->d_err);
        k_loss<<<dim3(P, kLossSplit), kLossThreads, 0, st>>>(P, ds->S, n_par, nullptr, ds->s_inv_na, ds->s_vtar,
                                                             ds->partials, ds->e_tar, z_pop, lam[0], lam[1], lam[2],
                                                             lam[3], lam[4], loss_inv(ds->S, ds->N, n_par), loss);
        return cuda_fail(cudaGetLastError(), "population evaluation kernels");
    }
    const int C = ds->n_chunks;
    const int W = std::max(1, std::min(std::min(sh.waves, kMaxWaves), C));
    // range ends: structure boundaries (the owner pass writes into the slots
    // of every atom of its structure), near equal shares of the pairs
    int ends[kMaxWaves];
    int n_ranges = 0;
    {
        const std::vector<int>& s0 = ds->h_schunk0;  // first chunk of each structure, then C
        const long long tot = ds->h_cpairs[C];
        int c_lo = 0;
        for (int w = 1; w <= W && c_lo < C; ++w) {
            int c_hi = C;
            if (w < W) {
                const long long target = tot * w / W;
                size_t k = 0;
                while (k < s0.size() && (s0[k] <= c_lo || ds->h_cpairs[s0[k]] < target)) ++k;
                c_hi = k < s0.size() ? s0[k] : C;
            }
            ends[n_ranges++] = c_hi;
            c_lo = c_hi;
        }
    }
    if (n_ranges == 1) {
        launch_contraction(ds, P, Pst, 0, C, st, st, false, nullptr, precision == NEP_PREC_BF16);
    } else {
        int c_lo = 0;
        for (int w = 0; w < n_ranges; ++w) {
            launch_contraction(ds, P, Pst, c_lo, ends[w], st, ds->aux, true, ds->ev_wave[w], precision == NEP_PREC_BF16);
            c_lo = ends[w];
        }
        cudaEventRecord(ds->ev_join, ds->aux);
        cudaStreamWaitEvent(st, ds->ev_join, 0);
    }
    k_loss<<<dim3(P, kLossSplit), kLossThreads, 0, st>>>(P, ds->S, n_par, ds->s_chunk0, ds->s_inv_na, ds->s_vtar,
                                                         ds->partials, ds->e_tar, z_pop, lam[0], lam[1], lam[2], lam[3],
                                                         lam[4], loss_inv(ds->S, ds->N, n_par), loss);
    return cuda_fail(cudaGetLastError(), "population evaluation kernels");
}

int evaluate(nep_model* m, nep_dataset* ds, const float* z_pop, int P, int precision, const double* lambdas,
             double* loss, cudaStream_t st)
{
    int rc = prepare_evaluation(ds, P);
    if (rc) return rc;
    return enqueue_evaluation(m, ds, z_pop, P, precision, lambdas, loss, st);
}

// Launches of one SNES generation: draws (or the given r), z = m + s r, the
// population evaluation, ranking and update.  Capturable after
// prepare_evaluation.
int enqueue_generation(snes_state* st, nep_dataset* ds, int precision, const double* lambdas, const float* r_in,
                       const SnesCtl* ctl, cudaStream_t cs)
{
    const long long tot = (long long)st->P * st->n_par;
    if (r_in) {
        int rc = cuda_fail(cudaMemcpyAsync(st->r, r_in, sizeof(float) * tot, cudaMemcpyDeviceToDevice, cs), "copy r");
        if (rc) return rc;
        k_make_pop<<<blocks_for(tot, 256), 256, 0, cs>>>(tot, st->n_par, st->mean, st->sigma, st->r, st->z);
    } else if (precision == NEP_PREC_BF16) {
        // the draws, z and the tensor-core records in one launch
        int rc = launch_pack_tc_draw(st->P, st->m->hp.n_neu, st->seed, st->d_gen, st->mean, st->sigma, st->r, st->z,
                                     ds->packed, cs);
        if (rc) return rc;
    } else {
        k_gauss<<<blocks_for((tot + 3) / 4, 256), 256, 0, cs>>>(tot, st->n_par, st->seed, st->d_gen, st->mean,
                                                                st->sigma, st->r, st->z);
    }
    const bool prepacked = !r_in && precision == NEP_PREC_BF16;
    int rc = enqueue_evaluation(st->m, ds, st->z, st->P, precision, lambdas, st->loss, cs, prepacked);
    if (rc) return rc;
    const float eta_s = (float)((3.0 + std::log((double)st->n_par)) / (5.0 * std::sqrt((double)st->n_par)));
    k_snes_update<<<blocks_for(st->n_par, kUpdateThreads), kUpdateThreads, 0, cs>>>(
        st->P, st->n_par, st->loss, st->util, st->r, st->mean, st->sigma, 1.f, eta_s, st->order, st->d_gen, ctl);
    return cuda_fail(cudaGetLastError(), "snes generation kernels");
}

}  // namespace

extern "C" {

int nep_dataset_create(nep_model* m, int n_struct, const int* n_atoms, const double* boxes, const double* pos,
                       const double* e_tar, const double* f_tar, const double* w_tar, nep_dataset** out)
{
    return nep_dataset_create_species(m, n_struct, n_atoms, boxes, pos, nullptr, e_tar, f_tar, w_tar, out);
}

int nep_dataset_create_species(nep_model* m, int n_struct, const int* n_atoms, const double* boxes,
                               const double* pos, const double* z_atom, const double* e_tar, const double* f_tar,
                               const double* w_tar, nep_dataset** out)
{
    if (!m || !n_atoms || !boxes || !pos || !e_tar || !f_tar || !w_tar || !out || n_struct < 1) {
        set_error("nep_dataset_create: NULL argument or no structures");
        return NEP_ERR_ARG;
    }
    if (!sizes_default(m->hp)) {
        set_error("nep_dataset_create: training sets have kernels for the 32-descriptor model only");
        return NEP_ERR_UNSUPPORTED;
    }
    *out = nullptr;
    long long Nl = 0;
    for (int s = 0; s < n_struct; ++s) {
        if (n_atoms[s] < 1) {
            set_error("nep_dataset_create: structure %d has no atoms", s);
            return NEP_ERR_ARG;
        }
        Nl += n_atoms[s];
    }
    if (Nl > kMaxAtoms) {
        set_error("nep_dataset_create: too many atoms");
        return NEP_ERR_ARG;
    }
    const int N = (int)Nl, S = n_struct;
    const double rmax = m->hp.rc_R > m->hp.rc_A ? m->hp.rc_R : m->hp.rc_A;
    std::vector<Box> hbox(S);
    for (int s = 0; s < S; ++s) {
        int rc = setup_box(boxes + 9 * s, rmax, hbox[s]);
        if (rc) return rc;
        hbox[s].nc[0] = hbox[s].nc[1] = hbox[s].nc[2] = 0;
    }
    std::vector<int> hsid(N), hsstart(S + 1), hnat(S), hchunk0(S + 1), hcb, hce;
    hsstart[0] = 0;
    for (int s = 0; s < S; ++s) {
        hsstart[s + 1] = hsstart[s] + n_atoms[s];
        hnat[s] = n_atoms[s];
        for (int i = hsstart[s]; i < hsstart[s + 1]; ++i) hsid[i] = s;
        hchunk0[s] = (int)hcb.size();
        for (int b = hsstart[s]; b < hsstart[s + 1]; b += kChunkAtoms) {
            hcb.push_back(b);
            hce.push_back(std::min(b + kChunkAtoms, hsstart[s + 1]));
        }
    }
    hchunk0[S] = (int)hcb.size();
    std::vector<double> hpos((size_t)3 * N);
    for (int i = 0; i < N; ++i)
        for (int d = 0; d < 3; ++d) hpos[(size_t)d * N + i] = pos[(size_t)3 * i + d];
    std::vector<float> hf((size_t)3 * N);
    for (size_t e = 0; e < hf.size(); ++e) hf[e] = (float)f_tar[e];
    std::vector<float> hz;
    if (z_atom) {
        hz.resize((size_t)N);
        for (int i = 0; i < N; ++i) {
            if (!(z_atom[i] > 0.0) || !std::isfinite(z_atom[i])) {
                set_error("nep_dataset_create_species: the species number of atom %d is not positive", i);
                return NEP_ERR_ARG;
            }
            hz[(size_t)i] = (float)z_atom[i];
        }
    }

    nep_dataset* ds = new (std::nothrow) nep_dataset();
    if (!ds) {
        set_error("nep_dataset_create: host allocation failed");
        return NEP_ERR_OOM;
    }
    ds->m = m;
    ds->S = S;
    ds->N = N;
    ds->uid = ++g_dataset_uid;
    ds->n_chunks = (int)hcb.size();
    long long* bytes = &ds->bytes;
    double* dpos = nullptr;
    float* dz = nullptr;
    ds->typed = z_atom ? 1 : 0;
    float*& xh = ds->xh;
    float*& xl = ds->xl;
    int *tmp = nullptr, *cnt = nullptr, *cnta = nullptr;
    long long*& rev = ds->rev;
    int rc = NEP_OK;
    auto fail = [&](int code) {
        dfree(dpos);
        dfree(dz);
        dfree(tmp);
        dfree(cnt);
        dfree(cnta);
        nep_dataset_destroy(ds);
        return code;
    };
    if ((rc = dalloc(&ds->boxes, S, bytes)) || (rc = dalloc(&ds->sid, N, bytes)) ||
        (rc = dalloc(&ds->sstart, S + 1, bytes)) || (rc = dalloc(&ds->s_natoms, S, bytes)) ||
        (rc = dalloc(&ds->s_inv_na, S, bytes)) || (rc = dalloc(&ds->s_vtar, (size_t)8 * S, bytes)) ||
        (rc = dalloc(&ds->s_chunk0, S + 1, bytes)) || (rc = dalloc(&ds->s_order, S, bytes)) ||
        (rc = dalloc(&ds->chunk_begin, ds->n_chunks, bytes)) ||
        (rc = dalloc(&ds->chunk_end, ds->n_chunks, bytes)) || (rc = dalloc(&ds->q, (size_t)N * kNdes, bytes)) ||
        (rc = dalloc(&ds->B, (size_t)N * kNdes * 3, bytes)) || (rc = dalloc(&ds->pstart, (size_t)N + 1, bytes)) ||
        (rc = dalloc(&ds->e_tar, S, bytes)) || (rc = dalloc(&ds->f_tar, (size_t)3 * N, bytes)) ||
        (rc = dalloc(&ds->w_tar, (size_t)6 * S, bytes)) || (rc = dalloc(&dpos, (size_t)3 * N, nullptr)) ||
        (rc = dalloc(&xh, (size_t)4 * N, nullptr)) || (rc = dalloc(&xl, (size_t)4 * N, nullptr)) ||
        (rc = dalloc(&tmp, (size_t)N * kDsCap, nullptr)) || (rc = dalloc(&cnt, N, nullptr)) ||
        (rc = dalloc(&cnta, N, nullptr)) || (z_atom && (rc = dalloc(&dz, N, nullptr))))
        return fail(rc);
    cudaError_t e = cudaSuccess;
    auto up = [&](void* dst, const void* src, size_t b) {
        if (e == cudaSuccess) e = cudaMemcpy(dst, src, b, cudaMemcpyHostToDevice);
    };
    up(ds->boxes, hbox.data(), sizeof(Box) * S);
    up(ds->sid, hsid.data(), sizeof(int) * N);
    up(ds->sstart, hsstart.data(), sizeof(int) * (S + 1));
    up(ds->s_natoms, hnat.data(), sizeof(int) * S);
    std::vector<double> hinv(S);
    for (int t = 0; t < S; ++t) hinv[t] = 1.0 / hnat[t];
    up(ds->s_inv_na, hinv.data(), sizeof(double) * S);
    // the virial targets and 1 / atoms in FP32 for the loss kernel's FP32
    // virial residuals: [S][8] = W_tar (6), 1 / atoms, 0
    std::vector<float> hvt((size_t)8 * S, 0.f);
    for (int t = 0; t < S; ++t) {
        for (int w = 0; w < 6; ++w) hvt[(size_t)8 * t + w] = (float)w_tar[(size_t)6 * t + w];
        hvt[(size_t)8 * t + 6] = (float)hinv[t];
    }
    up(ds->s_vtar, hvt.data(), sizeof(float) * hvt.size());
    up(ds->s_chunk0, hchunk0.data(), sizeof(int) * (S + 1));
    // fused contraction: blocks of the largest structures first (they take
    // longest), and the shared memory its largest structure needs
    std::vector<int> horder(S);
    for (int t = 0; t < S; ++t) horder[t] = t;
    std::stable_sort(horder.begin(), horder.end(), [&](int a, int b) { return hnat[a] > hnat[b]; });
    up(ds->s_order, horder.data(), sizeof(int) * S);
    ds->amax = hnat[horder[0]];
    ds->shape.fused = fused_fits(ds, 8) ? 8 : (fused_fits(ds, 4) ? 4 : 0);

    up(ds->chunk_begin, hcb.data(), sizeof(int) * hcb.size());
    up(ds->chunk_end, hce.data(), sizeof(int) * hce.size());
    up(dpos, hpos.data(), sizeof(double) * hpos.size());
    if (z_atom) up(dz, hz.data(), sizeof(float) * hz.size());
    up(ds->e_tar, e_tar, sizeof(double) * S);
    up(ds->f_tar, hf.data(), sizeof(float) * hf.size());
    up(ds->w_tar, w_tar, sizeof(double) * 6 * S);
    if (e != cudaSuccess) return fail(cuda_fail(e, "dataset upload"));

    const float rc2 = (float)(rmax * rmax), rcA2 = (float)(m->hp.rc_A * m->hp.rc_A);
    const float rcR2 = (float)(m->hp.rc_R * m->hp.rc_R);
    k_ds_split<<<blocks_for(N, 256), 256>>>(N, dpos, ds->sid, ds->boxes, dz, xh, xl, m->d_err);
    k_ds_list<<<blocks_for(N, 128), 128>>>(N, ds->sid, ds->sstart, ds->boxes, xh, xl, rc2, rcA2, tmp, cnt, cnta,
                                           m->d_err);
    if ((rc = cuda_fail(cudaDeviceSynchronize(), "dataset neighbour search"))) return fail(rc);
    unsigned bits = 0;
    cudaMemcpy(&bits, m->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (bits) {
        cudaMemset(m->d_err, 0, sizeof(unsigned));
        return fail(status_from_bits(bits));
    }
    std::vector<int> hc(N), hca(N);
    cudaMemcpy(hc.data(), cnt, sizeof(int) * N, cudaMemcpyDeviceToHost);
    cudaMemcpy(hca.data(), cnta, sizeof(int) * N, cudaMemcpyDeviceToHost);
    std::vector<long long> hps(N + 1), has(N + 1);
    hps[0] = has[0] = 0;
    for (int i = 0; i < N; ++i) {
        hps[i + 1] = hps[i] + hc[i];
        has[i + 1] = has[i] + hca[i];
    }
    ds->n_pairs = hps[N];
    ds->n_ang = has[N];
    ds->h_cb = hcb;
    ds->h_ce = hce;
    ds->h_schunk0 = hchunk0;
    ds->h_cpairs.resize(hcb.size() + 1);
    for (size_t c = 0; c < hcb.size(); ++c) ds->h_cpairs[c] = hps[hcb[c]];
    ds->h_cpairs[hcb.size()] = hps[N];
    long long*& dastart = ds->astart;
    if ((rc = dalloc(&ds->pj, (size_t)ds->n_pairs, bytes)) || (rc = dalloc(&ds->aidx, (size_t)ds->n_pairs, bytes)) ||
        (rc = dalloc(&ds->rec, (size_t)ds->n_pairs, bytes)) ||
        (rc = dalloc(&ds->ang, (size_t)ds->n_ang * kNA * kLmax * 3, bytes)) ||
        (rc = dalloc(&rev, (size_t)ds->n_pairs, bytes)) || (rc = dalloc(&dastart, (size_t)N + 1, bytes)))
        return fail(rc);
    up(ds->pstart, hps.data(), sizeof(long long) * (N + 1));
    up(dastart, has.data(), sizeof(long long) * (N + 1));
    if (e != cudaSuccess) return fail(cuda_fail(e, "dataset upload"));
    k_ds_sort<<<blocks_for(N, 128), 128>>>(N, ds->sid, ds->boxes, xh, xl, cnt, tmp);
    k_ds_compact<<<blocks_for(N, 128), 128>>>(N, tmp, ds->pstart, dastart, ds->sid, ds->boxes, xh, xl, rcA2, ds->pj,
                                              ds->aidx);
    k_ds_reverse<<<blocks_for(N, 128), 128>>>(N, ds->pstart, ds->pj, rev, m->d_err);
    k_ds_site<<<blocks_for(N, 64), 64>>>(N, ds->sid, ds->boxes, xh, xl, ds->pstart, ds->pj, ds->aidx, rcR2,
                                         rcA2, (float)m->hp.rc_R, (float)m->hp.rc_A, (float)(1.0 / m->hp.rc_R),
                                         (float)(1.0 / m->hp.rc_A), ds->typed, ds->q, ds->B, ds->rec, ds->ang);
    if (!rc && !(rc = dalloc(&ds->qpack, pop_tc_qpack_bytes(N), bytes)))
        rc = launch_pack_q_tc(N, ds->q, ds->qpack, nullptr);
    // tiles of the tensor-core owner pass: per owner a first tile with up to
    // kOwnerTcPairs pairs and the own-term and virial rows, further tiles of
    // up to kOwnerTcMorePairs pairs
    if (!rc) {
        std::vector<OwnerTile> ht;
        ds->h_tile0.assign((size_t)N + 1, 0);
        long long row0 = 0;
        for (int j = 0; j < N; ++j) {
            ds->h_tile0[j] = (int)ht.size();
            long long q = hps[j];
            bool first = true;
            do {
                const int cap = first ? kOwnerTcPairs : kOwnerTcMorePairs;
                OwnerTile T;
                T.j = j;
                T.nt = (int)std::min<long long>(cap, hps[j + 1] - q);
                T.extra = first ? 1 : 0;
                const int rows = 3 * T.nt + (first ? 9 : 0);
                T.groups = (rows + 7) / 8;
                T.q0 = q;
                T.row0 = row0;
                row0 += 8 * T.groups;
                q += T.nt;
                first = false;
                ht.push_back(T);
            } while (q < hps[j + 1]);
        }
        ds->h_tile0[N] = (int)ht.size();
        ds->n_tiles = (int)ht.size();
        if ((rc = dalloc(&ds->tiles, ht.size(), bytes)) || (rc = dalloc(&ds->apack, (size_t)row0 * 64, bytes)) ||
            (rc = dalloc(&ds->rowscale, (size_t)row0, bytes)))
            return fail(rc);
        up(ds->tiles, ht.data(), sizeof(OwnerTile) * ht.size());
        if (e != cudaSuccess) return fail(cuda_fail(e, "dataset upload"));
        rc = launch_pack_owner_tc(ds->n_tiles, ds->tiles, ds->rec, ds->aidx, ds->ang, ds->B, ds->pstart, ds->apack,
                                  ds->rowscale, nullptr);
    }
    if (!rc) rc = cuda_fail(cudaDeviceSynchronize(), "dataset precompute");
    if (rc) return fail(rc);
    cudaMemcpy(&bits, m->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (bits) {
        cudaMemset(m->d_err, 0, sizeof(unsigned));
        return fail(status_from_bits(bits));
    }
    dfree(dpos);
    dfree(dz);
    dfree(tmp);
    dfree(cnt);
    dfree(cnta);
    *out = ds;
    return NEP_OK;
}

int nep_dataset_destroy(nep_dataset* ds)
{
    if (!ds) return NEP_OK;
    cudaDeviceSynchronize();
    dfree(ds->boxes);
    dfree(ds->sid);
    dfree(ds->sstart);
    dfree(ds->s_natoms);
    dfree(ds->s_inv_na);
    dfree(ds->s_vtar);
    dfree(ds->s_chunk0);
    dfree(ds->s_order);
    dfree(ds->astart);
    dfree(ds->chunk_begin);
    dfree(ds->chunk_end);
    dfree(ds->q);
    dfree(ds->xh);
    dfree(ds->xl);
    dfree(ds->B);
    dfree(ds->pstart);
    dfree(ds->pj);
    dfree(ds->rev);
    dfree(ds->aidx);
    dfree(ds->rec);
    dfree(ds->ang);
    dfree(ds->e_tar);
    dfree(ds->f_tar);
    dfree(ds->w_tar);
    dfree(ds->W1t);
    dfree(ds->b1t);
    dfree(ds->w2t);
    dfree(ds->b2t);
    dfree(ds->G);
    dfree(ds->U);
    dfree(ds->partials);
    dfree(ds->packed);
    dfree(ds->qpack);
    dfree(ds->pbuf);
    dfree(ds->w6);
    dfree(ds->fown);
    dfree(ds->tiles);
    dfree(ds->apack);
    dfree(ds->rowscale);
    free_adjoint(ds->adj);
    for (int w = 0; w < kMaxWaves; ++w)
        if (ds->ev_wave[w]) cudaEventDestroy(ds->ev_wave[w]);
    if (ds->ev_join) cudaEventDestroy(ds->ev_join);
    if (ds->aux) cudaStreamDestroy(ds->aux);
    delete ds;
    return NEP_OK;
}

int nep_dataset_info(const nep_dataset* ds, int* n_atoms, long long* n_pairs, long long* device_bytes)
{
    if (!ds) {
        set_error("nep_dataset_info: NULL handle");
        return NEP_ERR_ARG;
    }
    if (n_atoms) *n_atoms = ds->N;
    if (n_pairs) *n_pairs = ds->n_pairs;
    if (device_bytes) *device_bytes = ds->bytes;
    return NEP_OK;
}

int nep_dataset_counts(const nep_dataset* ds, long long* counts)
{
    if (!ds || !counts) {
        set_error("nep_dataset_counts: NULL argument");
        return NEP_ERR_ARG;
    }
    counts[0] = ds->N;
    counts[1] = ds->n_pairs;
    counts[2] = ds->n_ang;
    counts[3] = ds->S;
    counts[4] = ds->amax;
    return NEP_OK;
}

int nep_dataset_descriptors(const nep_dataset* ds, float* q, void* stream)
{
    if (!ds || !q) {
        set_error("nep_dataset_descriptors: NULL argument");
        return NEP_ERR_ARG;
    }
    return cuda_fail(cudaMemcpyAsync(q, ds->q, sizeof(float) * (size_t)ds->N * kNdes, cudaMemcpyDeviceToDevice,
                                     (cudaStream_t)stream),
                     "copy descriptors");
}

int snes_evaluate_population(nep_model* m, nep_dataset* ds, const float* z_pop, int n_pop, int precision,
                             const double* lambdas, double* loss, void* stream)
{
    if (!m || !ds || ds->m != m || !z_pop || !loss || n_pop < 1 || n_pop > kMaxPop) {
        set_error("snes_evaluate_population: bad arguments (1 <= n_pop <= %d, dataset of this model)", kMaxPop);
        return NEP_ERR_ARG;
    }
    return evaluate(m, ds, z_pop, n_pop, precision, lambdas, loss, (cudaStream_t)stream);
}

int snes_create(nep_model* m, int n_pop, const float* mean0, const float* sigma0, unsigned long long seed,
                snes_state** out)
{
    if (!m || !mean0 || !sigma0 || !out || n_pop < 2 || n_pop > kMaxPop) {
        set_error("snes_create: bad arguments (2 <= n_pop <= %d)", kMaxPop);
        return NEP_ERR_ARG;
    }
    *out = nullptr;
    snes_state* st = new (std::nothrow) snes_state();
    if (!st) {
        set_error("snes_create: host allocation failed");
        return NEP_ERR_OOM;
    }
    st->m = m;
    st->P = n_pop;
    st->n_par = m->n_par;
    st->seed = seed;
    const size_t np = (size_t)m->n_par, tot = np * n_pop;
    int rc;
    if ((rc = dalloc(&st->mean, np, nullptr)) || (rc = dalloc(&st->sigma, np, nullptr)) ||
        (rc = dalloc(&st->r, tot, nullptr)) || (rc = dalloc(&st->z, tot, nullptr)) ||
        (rc = dalloc(&st->loss, (size_t)n_pop * 6, nullptr)) || (rc = dalloc(&st->order, (size_t)n_pop, nullptr)) ||
        (rc = dalloc(&st->util, (size_t)n_pop, nullptr)) || (rc = dalloc(&st->d_gen, 1, nullptr)) ||
        (rc = dalloc(&st->d_ctl, 1, nullptr))) {
        snes_destroy(st);
        return rc;
    }
    // rank utilities (standard NES rank shaping, Sec. II.D.2):
    // u_q = max(0, ln(P/2 + 1) - ln q) / sum_q' max(0, ln(P/2 + 1) - ln q') - 1/P
    std::vector<float> util(n_pop);
    {
        const double top = std::log(n_pop / 2.0 + 1.0);
        double sum = 0.0;
        for (int q = 1; q <= n_pop; ++q) sum += std::fmax(0.0, top - std::log((double)q));
        for (int q = 1; q <= n_pop; ++q)
            util[q - 1] = (float)(std::fmax(0.0, top - std::log((double)q)) / sum - 1.0 / n_pop);
    }
    cudaError_t e = cudaMemcpy(st->mean, mean0, sizeof(float) * np, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(st->sigma, sigma0, sizeof(float) * np, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(st->util, util.data(), sizeof(float) * n_pop, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(st->d_gen, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(st->d_ctl, 0, sizeof(SnesCtl));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        snes_destroy(st);
        return cuda_fail(e, "snes_create upload");
    }
    *out = st;
    return NEP_OK;
}

int snes_destroy(snes_state* st)
{
    if (!st) return NEP_OK;
    cudaDeviceSynchronize();
    dfree(st->mean);
    dfree(st->sigma);
    dfree(st->r);
    dfree(st->z);
    dfree(st->loss);
    dfree(st->order);
    dfree(st->util);
    dfree(st->d_gen);
    dfree(st->d_ctl);
    if (st->exec) cudaGraphExecDestroy(st->exec);
    if (st->cap) cudaStreamDestroy(st->cap);
    delete st;
    return NEP_OK;
}

int snes_step(snes_state* st, nep_dataset* ds, int precision, const double* lambdas, const float* r_in,
              double* loss_out, void* stream)
{
    if (!st || !ds || ds->m != st->m) {
        set_error("snes_step: bad arguments");
        return NEP_ERR_ARG;
    }
    cudaStream_t cs = (cudaStream_t)stream;
    int rc = prepare_evaluation(ds, st->P);
    if (rc) return rc;
    if ((rc = enqueue_generation(st, ds, precision, lambdas, r_in, nullptr, cs))) return rc;
    if (loss_out) {
        rc = cuda_fail(cudaMemcpyAsync(loss_out, st->loss, sizeof(double) * st->P * 6, cudaMemcpyDeviceToDevice, cs),
                       "copy loss");
        if (rc) return rc;
    }
    ++st->gen;
    return NEP_OK;
}

int snes_run(snes_state* st, nep_dataset* ds, int precision, const double* lambdas, int n_gen, double* loss_hist,
             void* stream)
{
    if (!st || !ds || ds->m != st->m || n_gen < 0) {
        set_error("snes_run: bad arguments (dataset of this model, n_gen >= 0)");
        return NEP_ERR_ARG;
    }
    if (precision != NEP_PREC_FP32 && precision != NEP_PREC_BF16) {
        set_error("snes_run: unknown precision %d", precision);
        return NEP_ERR_ARG;
    }
    if (n_gen == 0) return NEP_OK;
    cudaStream_t cs = (cudaStream_t)stream;
    int rc = prepare_evaluation(ds, st->P);
    if (rc) return rc;
    double lam[5] = {1.0, 1.0, 1.0, 0.05, 0.05};
    if (lambdas)
        for (int k = 0; k < 5; ++k) lam[k] = lambdas[k];
    bool same = st->exec && st->key_uid == ds->uid && st->key_epoch == ds->epoch && st->key_prec == precision;
    for (int k = 0; same && k < 5; ++k) same = st->key_lam[k] == lam[k];
    if (!same) {
        if (st->exec) cudaGraphExecDestroy(st->exec);
        st->exec = nullptr;
        cudaGraph_t g = nullptr;
        if ((rc = cuda_fail(cudaStreamBeginCapture(st->cap, cudaStreamCaptureModeThreadLocal), "begin capture")))
            return rc;
        rc = enqueue_generation(st, ds, precision, lam, nullptr, st->d_ctl, st->cap);
        const cudaError_t e = cudaStreamEndCapture(st->cap, &g);
        if (!rc && e != cudaSuccess) rc = cuda_fail(e, "end capture");
        if (!rc) rc = cuda_fail(cudaGraphInstantiate(&st->exec, g, 0), "instantiate generation graph");
        if (g) cudaGraphDestroy(g);
        if (rc) {
            st->exec = nullptr;
            return rc;
        }
        st->key_uid = ds->uid;
        st->key_epoch = ds->epoch;
        st->key_prec = precision;
        for (int k = 0; k < 5; ++k) st->key_lam[k] = lam[k];
    }
    k_set_ctl<<<1, 1, 0, cs>>>(st->d_ctl, loss_hist, st->gen);
    for (int g = 0; g < n_gen; ++g)
        if ((rc = cuda_fail(cudaGraphLaunch(st->exec, cs), "launch generation graph"))) return rc;
    k_set_ctl<<<1, 1, 0, cs>>>(st->d_ctl, nullptr, 0u);
    st->gen += (unsigned)n_gen;
    return cuda_fail(cudaGetLastError(), "snes_run");
}

int nep_dataset_set_shape(nep_dataset* ds, const int* shape)
{
    if (!ds || !shape) {
        set_error("nep_dataset_set_shape: NULL argument");
        return NEP_ERR_ARG;
    }
    EvalShape h;
    h.waves = shape[0];
    h.owner_warps = shape[1];
    h.discard = shape[2];
    h.mlp_threads = shape[3];
    h.recv_unroll = shape[4];
    h.fused = shape[5];
    h.owner_tc = shape[6];
    h.pop_pipe = shape[7];
    if (!valid_shape(ds, h)) {
        set_error("nep_dataset_set_shape: waves 1..%d, owner warps 4 or 8, discard 0 or 1, network threads 128 or 256, "
                  "receiver unroll 4, 8, 12, 16 (staged) or 1 (bulk copies), fused 0, 4, 8 or 16 members per block (%d atoms x members x "
                  "48 bytes of shared memory at most %zu), owner_tc 0 or 1, pop_pipe 0 or 1",
                  kMaxWaves, ds->amax, kFusedSmemMax);
        return NEP_ERR_ARG;
    }
    ds->shape = h;
    ++ds->epoch;
    return NEP_OK;
}

int nep_dataset_get_shape(const nep_dataset* ds, int* shape)
{
    if (!ds || !shape) {
        set_error("nep_dataset_get_shape: NULL argument");
        return NEP_ERR_ARG;
    }
    shape[0] = ds->shape.waves;
    shape[1] = ds->shape.owner_warps;
    shape[2] = ds->shape.discard;
    shape[3] = ds->shape.mlp_threads;
    shape[4] = ds->shape.recv_unroll;
    shape[5] = ds->shape.fused;
    shape[6] = ds->shape.owner_tc;
    shape[7] = ds->shape.pop_pipe;
    return NEP_OK;
}

int nep_dataset_tune(nep_model* m, nep_dataset* ds, int n_pop, int precision, int reps, int* shape_out,
                     float* ms_out, void* stream)
{
    if (!m || !ds || ds->m != m || n_pop < 1 || n_pop > kMaxPop || reps < 1 ||
        (precision != NEP_PREC_FP32 && precision != NEP_PREC_BF16)) {
        set_error("nep_dataset_tune: bad arguments (dataset of this model, 1 <= n_pop <= %d, reps >= 1)", kMaxPop);
        return NEP_ERR_ARG;
    }
    cudaStream_t cs = (cudaStream_t)stream;
    int rc = prepare_evaluation(ds, n_pop);
    if (rc) return rc;
    std::vector<EvalShape> cand;
    const int wv[] = {1, 2, 4};
    for (int w : wv)
        for (int ow = 4; ow <= 8; ow += 4)
            for (int dc = 0; dc <= 1; ++dc)
                for (int mt = 128; mt <= 256; mt += 128)
                    for (int ru : {1, 4, 8, 12, 16}) {
                        if (precision == NEP_PREC_BF16 && mt == 128) continue;  // the FP32 network is not launched
                        EvalShape h;
                        h.waves = w;
                        h.owner_warps = ow;
                        h.discard = dc;
                        h.mlp_threads = mt;
                        h.recv_unroll = ru;
                        // BF16: the network as the pipelined persistent kernel or not,
                        // and the owner pass on the tensor cores (owner warps do not apply)
                        for (int pp = 0; pp <= (precision == NEP_PREC_BF16 ? 1 : 0); ++pp) {
                            h.pop_pipe = pp;
                            h.owner_tc = 0;
                            cand.push_back(h);
                            if (precision == NEP_PREC_BF16 && ow == 4) {
                                h.owner_tc = 1;
                                cand.push_back(h);
                            }
                        }
                    }
    // the fused contraction: members per block (the atoms per warp follow:
    // 32 / members), with the FP32 network's block size where it runs
    for (int gm = 4; gm <= 16; gm *= 2)
        for (int mt = 128; mt <= 256; mt += 128) {
            if (!fused_fits(ds, gm) || (precision == NEP_PREC_BF16 && mt == 128)) continue;
            EvalShape h;
            h.mlp_threads = mt;
            h.fused = gm;
            for (int pp = 0; pp <= (precision == NEP_PREC_BF16 ? 1 : 0); ++pp) {
                h.pop_pipe = pp;
                cand.push_back(h);
            }
        }
    const long long tot = (long long)n_pop * m->n_par;
    float* z = nullptr;
    double* loss = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const EvalShape keep = ds->shape;
    auto cleanup = [&](int code) {
        dfree(z);
        dfree(loss);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        return code;
    };
    if ((rc = dalloc(&z, (size_t)tot, nullptr)) || (rc = dalloc(&loss, (size_t)n_pop * 6, nullptr))) return cleanup(rc);
    if ((rc = cuda_fail(cudaEventCreate(&e0), "tune events")) || (rc = cuda_fail(cudaEventCreate(&e1), "tune events")))
        return cleanup(rc);
    k_tune_pop<<<blocks_for(tot, 256), 256, 0, cs>>>(tot, z);
    float best_ms = 0.f;
    EvalShape best = keep;
    for (size_t c = 0; c < cand.size(); ++c) {
        ds->shape = cand[c];
        rc = enqueue_evaluation(m, ds, z, n_pop, precision, nullptr, loss, cs);  // warm-up
        if (!rc) rc = cuda_fail(cudaEventRecord(e0, cs), "tune event");
        for (int r = 0; !rc && r < reps; ++r) rc = enqueue_evaluation(m, ds, z, n_pop, precision, nullptr, loss, cs);
        if (!rc) rc = cuda_fail(cudaEventRecord(e1, cs), "tune event");
        if (!rc) rc = cuda_fail(cudaEventSynchronize(e1), "tune timing");
        float ms = 0.f;
        if (!rc) rc = cuda_fail(cudaEventElapsedTime(&ms, e0, e1), "tune timing");
        if (rc) {
            ds->shape = keep;
            return cleanup(rc);
        }
        ms /= (float)reps;
        if (c == 0 || ms < best_ms) {
            best_ms = ms;
            best = cand[c];
        }
    }
    ds->shape = best;
    ++ds->epoch;
    if (shape_out) nep_dataset_get_shape(ds, shape_out);
    if (ms_out) *ms_out = best_ms;
    return cleanup(NEP_OK);
}

int snes_get_state(snes_state* st, float* mean, float* sigma, float* r_last, int* order, void* stream)
{
    if (!st) {
        set_error("snes_get_state: NULL handle");
        return NEP_ERR_ARG;
    }
    cudaStream_t cs = (cudaStream_t)stream;
    const size_t np = (size_t)st->n_par;
    cudaError_t e = cudaSuccess;
    if (mean) e = cudaMemcpyAsync(mean, st->mean, sizeof(float) * np, cudaMemcpyDeviceToDevice, cs);
    if (e == cudaSuccess && sigma) e = cudaMemcpyAsync(sigma, st->sigma, sizeof(float) * np, cudaMemcpyDeviceToDevice, cs);
    if (e == cudaSuccess && r_last)
        e = cudaMemcpyAsync(r_last, st->r, sizeof(float) * np * st->P, cudaMemcpyDeviceToDevice, cs);
    if (e == cudaSuccess && order) e = cudaMemcpyAsync(order, st->order, sizeof(int) * st->P, cudaMemcpyDeviceToDevice, cs);
    return cuda_fail(e, "snes_get_state");
}

}  // extern "C"
