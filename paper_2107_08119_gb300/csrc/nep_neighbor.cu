// nep_neighbor.cu -- cell binning and Verlet neighbour list on the device.
//
// The paper keeps neighbour lists of atoms within the cutoffs (Sec. III.C,
// "memory consumption") without describing their construction.  Here:
//   1. wrap positions into the orthorhombic box, split them into FP32 hi/lo,
//      bin atoms into cells of edge >= the list radius;
//   2. exclusive scan of the cell counts and scatter (the order of atoms
//      within a cell is whatever the atomics give: the list order below
//      depends only on the sort keys, so it stays deterministic);
//   3. one warp per atom scans the 27 neighbouring cells and keeps every
//      (j, image) with |r_ij| below the list radius (full list, both
//      directions), then orders its slots by increasing distance (the
//      partial-force buffer is free at this point and holds the sort keys,
//      atom-major: key[i * m_cap + k]; the values are also kept atom-major
//      in vala[i * m_cap + k] for the reverse search and the site pass);
//   4. the reverse-pair index: for slot k of atom i, the slot of i in j's
//      list, by binary search over j's contiguous keys.
// Boxes with fewer than 3 cells in a direction (small training cells) use a
// brute-force scan over all atoms and images instead of cells.
// Every kernel takes an optional device gate word: when it is zero the kernel
// returns at once, which lets the MD step skip the rebuild without a host
// round trip.
#include <algorithm>
#include <cstdio>

#include "nep_internal.cuh"

namespace nep {

namespace {

__device__ __forceinline__ bool gated_off(const unsigned* gate)
{
    return gate != nullptr && *((volatile const unsigned*)gate) == 0u;
}

// A non-finite coordinate latches kErrNonFinite: such an atom would
// otherwise be binned into a clamped cell and simply see no neighbours.
__global__ void k_bin(int n, double* __restrict__ pos, const float* __restrict__ zatom, int wrap_in_place,
                      double* __restrict__ x_ref, float* __restrict__ xh, float* __restrict__ xl,
                      int* __restrict__ atom_cell, int* __restrict__ cell_count, Box b, const unsigned* gate,
                      unsigned* __restrict__ err)
{
    if (gated_off(gate)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c[3];
    double wx[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double L = b.L[d];
        const double x = pos[(size_t)d * n + i];
        if (!isfinite(x)) atomicOr(err, kErrNonFinite);
        // FP64 division is slow here: atoms within one box length of the box
        // (all of them between MD rebuilds) wrap by one exact subtraction
        double w;
        if (x >= 0.0 && x < L)
            w = x;
        else if (x >= L && x < 2.0 * L)
            w = x - L;
        else if (x < 0.0 && x >= -L)
            w = x + L;
        else
            w = x - L * floor(x / L);
        if (w >= L) w -= L;
        if (w < 0.0) w = 0.0;
        if (wrap_in_place) {
            pos[(size_t)d * n + i] = w;
            if (x_ref) x_ref[(size_t)d * n + i] = w;
        }
        wx[d] = w;
        if (b.nc[0] > 0) {
            // any cell within rounding of the true one is valid (cells are at
            // least the list radius wide); the list order depends only on keys
            int ci = (int)(w * b.cpl[d]);
            c[d] = ci < 0 ? 0 : (ci >= b.nc[d] ? b.nc[d] - 1 : ci);
        }
    }
    store_pos(xh, xl, i, wx, zatom ? zatom[i] : 1.f);
    if (b.nc[0] > 0) {
        const int cid = (c[0] * b.nc[1] + c[1]) * b.nc[2] + c[2];
        atom_cell[i] = cid;
        atomicAdd(cell_count + cid, 1);
    }
}

// Single-block exclusive scan: cell_start[c] = sum_{c' < c} count[c'].  Also
// clears the per-cell counters for the scatter and the next build.  Rounds
// of blockDim * kScanPer cells go through shared memory (coalesced global
// reads and writes; padded so that a thread's run of kScanPer consecutive
// cells is conflict-free); warp shuffles and the warp totals give the prefix.
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 8;
constexpr int kScanRound = kScanThreads * kScanPer;

__device__ __forceinline__ int scan_pad(int x) { return x + (x >> 5); }

__global__ void __launch_bounds__(kScanThreads) k_scan(int ncell, int* __restrict__ count, int* __restrict__ start,
                                                       int* __restrict__ fill, const unsigned* gate)
{
    if (gated_off(gate)) return;
    __shared__ int sc[kScanRound + kScanRound / 32];
    __shared__ int wsum[kScanThreads / 32];
    __shared__ int carry;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) carry = 0;
    for (int base = 0; base < ncell; base += kScanRound) {
#pragma unroll
        for (int e = 0; e < kScanPer; ++e) {
            const int x = e * kScanThreads + t;
            sc[scan_pad(x)] = base + x < ncell ? count[base + x] : 0;
        }
        __syncthreads();
        int v[kScanPer];
        int s = 0;
#pragma unroll
        for (int e = 0; e < kScanPer; ++e) {
            v[e] = sc[scan_pad(t * kScanPer + e)];
            s += v[e];
        }
        int incl = s;  // inclusive scan of the thread sums within the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int w = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            wsum[lane] = w;  // inclusive over warps
        }
        __syncthreads();
        int run = carry + (warp > 0 ? wsum[warp - 1] : 0) + incl - s;
#pragma unroll
        for (int e = 0; e < kScanPer; ++e) {
            sc[scan_pad(t * kScanPer + e)] = run;
            run += v[e];
        }
        __syncthreads();  // every thread has read carry and wsum, and sc holds the prefixes
        if (t == kScanThreads - 1) carry = run;
#pragma unroll
        for (int e = 0; e < kScanPer; ++e) {
            const int x = e * kScanThreads + t;
            if (base + x < ncell) {
                start[base + x] = sc[scan_pad(x)];
                count[base + x] = 0;
                fill[base + x] = 0;
            }
        }
        __syncthreads();
    }
    if (t == 0) start[ncell] = carry;
}

__global__ void k_scatter(int n, const int* __restrict__ atom_cell, const int* __restrict__ cell_start,
                          int* __restrict__ cell_fill, int* __restrict__ cell_atoms, const unsigned* gate)
{
    if (gated_off(gate)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = atom_cell[i];
    const int slot = atomicAdd(cell_fill + c, 1);
    cell_atoms[cell_start[c] + slot] = i;
}

__device__ __forceinline__ void list_push(int i, int n, int m_cap, int& cnt, int value, float d2, int* __restrict__ nbr,
                                          float* __restrict__ key)
{
    if (cnt < m_cap) {
        nbr[(size_t)cnt * n + i] = value;
        key[(size_t)i * m_cap + cnt] = d2;
    }
    ++cnt;
}

// Order atom i's slots by increasing distance (insertion sort, stable).  Slot
// k then holds roughly the k-th nearest neighbour of every atom, so the lanes
// of a warp agree on which slots need the (long) angular work, and the force
// pass can add the nearest (largest) terms last by walking ranks downwards.
__device__ void sort_near_first(int i, int n, int m_cap, int cnt, int* __restrict__ nbr, float* __restrict__ key)
{
    float* ki = key + (size_t)i * m_cap;
    for (int a = 1; a < cnt; ++a) {
        const float kd = ki[a];
        const int kv = nbr[(size_t)a * n + i];
        int b = a - 1;
        while (b >= 0 && ki[b] > kd) {
            ki[b + 1] = ki[b];
            nbr[(size_t)(b + 1) * n + i] = nbr[(size_t)b * n + i];
            --b;
        }
        ki[b + 1] = kd;
        nbr[(size_t)(b + 1) * n + i] = kv;
    }
}

// One warp per atom.  The candidates of the 27 neighbouring cells are
// numbered consecutively (cell by cell) and the lanes take them 32 at a time
// (a lane finds its cell by stepping from the round's first cell); a quick
// test on the hi parts compacts the survivors with a ballot, the exact test
// then runs on them with every lane busy, and the accepted pairs are sorted
// by (squared distance, packed index) by ranking and written out.
// Sorting on the pair of keys makes the order unique, hence deterministic.
constexpr int kVerletWarps = 4;
constexpr int kVerletCellWords = 192;  // per-warp cell tables: prefix, start, code, 3 shifts (32 words each)

// (squared distance, packed index) as one unsigned 64-bit sort key: d2 >= 0,
// so its IEEE bits order like its value, and the packed index is below 2^31.
__device__ __forceinline__ unsigned long long sort_key(float d2, int v)
{
    return ((unsigned long long)__float_as_uint(d2) << 32) | (unsigned)v;
}

// Sorts the warp's accepted entries by their keys and writes the first m of
// them: lane l ranks the entries c0 + l + 32 t against all ns entries
// (broadcast shared-memory reads, one 64-bit compare each) and stores each
// at its rank, slot-major in nbr and atom-major in key / vala.  The pairs are
// distinct, so the ranks are a permutation.
template <int EPL>
__device__ __forceinline__ void rank_sort_write(int c0, int ns, int m, int lane, const unsigned long long* sk, int i,
                                                int n, int m_cap, int* __restrict__ nbr, float* __restrict__ key,
                                                int* __restrict__ vala)
{
    unsigned long long ke[EPL];
    int rk[EPL];
#pragma unroll
    for (int t = 0; t < EPL; ++t) {
        const int e = c0 + lane + 32 * t;
        ke[t] = e < ns ? sk[e] : ~0ull;
        rk[t] = 0;
    }
    for (int f = 0; f < ns; ++f) {
        const unsigned long long kf = sk[f];
#pragma unroll
        for (int t = 0; t < EPL; ++t) rk[t] += ke[t] > kf ? 1 : 0;
    }
#pragma unroll
    for (int t = 0; t < EPL; ++t) {
        const int e = c0 + lane + 32 * t;
        if (e < ns && rk[t] < m) {
            const int v = (int)(unsigned)ke[t];
            nbr[(size_t)rk[t] * n + i] = v;
            key[(size_t)i * m_cap + rk[t]] = __uint_as_float((unsigned)(ke[t] >> 32));
            vala[(size_t)i * m_cap + rk[t]] = v;
        }
    }
}

__global__ void __launch_bounds__(32 * kVerletWarps) k_verlet_cells(int n, int m_cap, int lcap, float rv2,
                                                                   const float* __restrict__ xh,
                                                                   const float* __restrict__ xl,
                                                                   const int* __restrict__ atom_cell,
                                                                   const int* __restrict__ cell_start,
                                                                   const int* __restrict__ cell_atoms,
                                                                   int* __restrict__ count, int* __restrict__ nbr,
                                                                   float* __restrict__ key, int* __restrict__ vala,
                                                                   unsigned* err, Box b, const unsigned* gate)
{
    if (gated_off(gate)) return;
    extern __shared__ float s_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // per warp: lcap sort keys, lcap quick-test survivors, 28 prefix sums,
    // 27 starts, 27 codes, 27 image shifts (x, y, z)
    unsigned long long* sk = reinterpret_cast<unsigned long long*>(s_raw + (size_t)warp * (3 * lcap + kVerletCellWords));
    int* sq = reinterpret_cast<int*>(sk + lcap);
    int* pre = sq + lcap;
    int* cst = pre + 32;
    int* ccode = cst + 32;
    float* csh = reinterpret_cast<float*>(ccode + 32);
    // a bounded grid strides over the atoms, so a gated-off launch is cheap
    for (int i = blockIdx.x * kVerletWarps + warp; i < n; i += gridDim.x * kVerletWarps) {
        float hi[3], li[3];
        load_pos(xh, xl, n, i, hi, li);
        const int cid = atom_cell[i];
        const int cz = cid % b.nc[2];
        const int cy = (cid / b.nc[2]) % b.nc[1];
        const int cx = cid / (b.nc[2] * b.nc[1]);
        // lane c < 27 describes neighbouring cell c (x slowest, z fastest)
        int ccount = 0;
        if (lane < 27) {
            int x2 = cx + lane / 9 - 1, y2 = cy + (lane / 3) % 3 - 1, z2 = cz + lane % 3 - 1;
            int sx = 0, sy = 0, sz = 0;
            if (x2 < 0) { x2 += b.nc[0]; sx = -1; } else if (x2 >= b.nc[0]) { x2 -= b.nc[0]; sx = 1; }
            if (y2 < 0) { y2 += b.nc[1]; sy = -1; } else if (y2 >= b.nc[1]) { y2 -= b.nc[1]; sy = 1; }
            if (z2 < 0) { z2 += b.nc[2]; sz = -1; } else if (z2 >= b.nc[2]) { z2 -= b.nc[2]; sz = 1; }
            const int c2 = (x2 * b.nc[1] + y2) * b.nc[2] + z2;
            const int c2s = cell_start[c2];
            ccount = cell_start[c2 + 1] - c2s;
            cst[lane] = c2s;
            ccode[lane] = image_code(sx, sy, sz);
            csh[lane] = (float)sx * b.Lh[0];  // exact: s in {-1, 0, 1}
            csh[32 + lane] = (float)sy * b.Lh[1];
            csh[64 + lane] = (float)sz * b.Lh[2];
        }
        // exclusive prefix of the cell sizes
        int incl = ccount;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane < 28) pre[lane] = incl - ccount;
        if (lane < 27) cst[lane] -= incl - ccount;  // candidate idx of cell c sits at cell_atoms[cst[c] + idx]
        __syncwarp();
        const int total = pre[27];
        // Pass 1, quick rejection with the hi parts only: their pair vector is
        // within 1e-4 A of the hi/lo one, so the 1e-3 A margin never drops a
        // pair that the exact test keeps.  Survivors are compacted into sq.
        const float rq = sqrtf(rv2) + 1e-3f, rq2 = rq * rq;
        int nq = 0;
        int c0 = 0;  // cell of this round's first candidate (warp-uniform)
        for (int base = 0; base < total; base += 32) {
            const int idx = base + lane;
            bool pass = false;
            int value = 0;
            int c = c0;
            if (idx < total) {
                while (pre[c + 1] <= idx) ++c;  // a cell holds ~12 atoms: 0-3 steps
                const int j = cell_atoms[cst[c] + idx];
                const int code = ccode[c];
                if (!(j == i && code == kImgCenter)) {
                    const float4 a = NEP_LDG(reinterpret_cast<const float4*>(xh) + j);
                    const float qx = (a.x - hi[0]) + csh[c];
                    const float qy = (a.y - hi[1]) + csh[32 + c];
                    const float qz = (a.z - hi[2]) + csh[64 + c];
                    pass = fmaf(qx, qx, fmaf(qy, qy, qz * qz)) < rq2;
                    value = j | (code << 24);
                }
            }
            c0 = __shfl_sync(0xffffffffu, c, 31);
            const unsigned mask = __ballot_sync(0xffffffffu, pass);
            const int pos = nq + __popc(mask & ((1u << lane) - 1u));
            if (pass && pos < lcap) sq[pos] = value;
            nq += __popc(mask);
        }
        __syncwarp();
        if (nq > lcap && lane == 0) atomicOr(err, kErrOverflow);
        // Pass 2, the exact (canonical hi/lo) test on the survivors, every
        // lane busy; accepted pairs are compacted into sk as sort keys.
        const int nqs = nq < lcap ? nq : lcap;
        int cnt = 0;
        for (int base = 0; base < nqs; base += 32) {
            const int e = base + lane;
            bool accept = false;
            int value = 0;
            float d2 = 0.f;
            if (e < nqs) {
                value = sq[e];
                const int j = value & 0xFFFFFF;
                float hj[3], lj[3];
                load_pos(xh, xl, n, j, hj, lj);
                float rx, ry, rz;
                pair_vector(i, j, value >> 24, hi, li, hj, lj, b, rx, ry, rz);
                d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                accept = d2 < rv2;
            }
            const unsigned mask = __ballot_sync(0xffffffffu, accept);
            const int pos = cnt + __popc(mask & ((1u << lane) - 1u));
            if (accept) sk[pos] = sort_key(d2, value);  // pos < nqs <= lcap
            cnt += __popc(mask);
        }
        __syncwarp();
        if (lane == 0) count[i] = cnt;
        if (cnt > m_cap && lane == 0) atomicOr(err, kErrOverflow);
        const int m = cnt < m_cap ? cnt : m_cap;
        const int ns = cnt < lcap ? cnt : lcap;
        if (ns <= 32)
            rank_sort_write<1>(0, ns, m, lane, sk, i, n, m_cap, nbr, key, vala);
        else if (ns <= 64)
            rank_sort_write<2>(0, ns, m, lane, sk, i, n, m_cap, nbr, key, vala);
        else
            for (int c0 = 0; c0 < ns; c0 += 128) rank_sort_write<4>(c0, ns, m, lane, sk, i, n, m_cap, nbr, key, vala);
        __syncwarp();  // the warp's buffers are reused by its next atom
    }
}

__global__ void k_verlet_brute(int n, int m_cap, float rv2, const float* __restrict__ xh,
                               const float* __restrict__ xl, int* __restrict__ count, int* __restrict__ nbr,
                               float* __restrict__ key, int* __restrict__ vala, unsigned* err, Box b,
                               const unsigned* gate)
{
    if (gated_off(gate)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float hi[3], li[3];
    load_pos(xh, xl, n, i, hi, li);
    int cnt = 0;
    for (int j = 0; j < n; ++j) {
        float hj[3], lj[3];
        load_pos(xh, xl, n, j, hj, lj);
        for (int sx = -b.img[0]; sx <= b.img[0]; ++sx)
            for (int sy = -b.img[1]; sy <= b.img[1]; ++sy)
                for (int sz = -b.img[2]; sz <= b.img[2]; ++sz) {
                    const int code = image_code(sx, sy, sz);
                    if (j == i && code == kImgCenter) continue;
                    float rx, ry, rz;
                    pair_vector(i, j, code, hi, li, hj, lj, b, rx, ry, rz);
                    const float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                    if (d2 < rv2) list_push(i, n, m_cap, cnt, j | (code << 24), d2, nbr, key);
                }
    }
    count[i] = cnt;
    if (cnt > m_cap) atomicOr(err, kErrOverflow);
    const int m = cnt < m_cap ? cnt : m_cap;
    sort_near_first(i, n, m_cap, m, nbr, key);
    for (int k = 0; k < m; ++k) vala[(size_t)i * m_cap + k] = nbr[(size_t)k * n + i];
}

// rev[k][i] = slot of (i, -image) in j's list.  The pair vectors are exactly
// antisymmetric, so both directions carry the same squared distance and j's
// list (sorted by it) is binary-searched; a miss (only possible after an
// overflow) is latched as an error.  One warp per atom, a lane per slot; the
// keys and values are read from their atom-major copies, so every search
// stays inside one atom's contiguous row.
__global__ void k_reverse(int n, int m_cap, const int* __restrict__ count, const float* __restrict__ key,
                          const int* __restrict__ vala, int* __restrict__ rev, unsigned* err, const unsigned* gate)
{
    if (gated_off(gate)) return;
    const int lane = threadIdx.x & 31;
    const int warps = (int)((gridDim.x * blockDim.x) >> 5);
    for (int i = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); i < n; i += warps) {
        const int ci = min(count[i], m_cap);
        for (int k = lane; k < ci; k += 32) {
            const int v = vala[(size_t)i * m_cap + k];
            const int j = v & 0xFFFFFF;
            const int target = i | ((124 - (v >> 24)) << 24);
            const float kd = key[(size_t)i * m_cap + k];
            const int cj = min(count[j], m_cap);
            const float* kj = key + (size_t)j * m_cap;  // j's keys, contiguous
            int lo = 0, hi = cj;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (kj[mid] < kd)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            int found = -1;
            for (int t = lo; t < cj && kj[t] == kd; ++t)
                if (vala[(size_t)j * m_cap + t] == target) {
                    found = t;
                    break;
                }
            if (found < 0) {
                atomicOr(err, kErrReverse);
                found = k;  // keeps later reads in bounds
            }
            rev[(size_t)k * n + i] = found;
        }
    }
}

inline int blocks_for(int n, int t) { return (n + t - 1) / t; }

// grid of the warp-per-atom list kernels: 152 SMs x 16 blocks of 4 warps
// keep every SM full, and a launch whose gate is off retires in microseconds
constexpr int kListGridCap = 152 * 16;

}  // namespace

int build_neighbor_list(NeighborList& nl, const Box& b, int n, double* pos, const float* zatom, bool wrap_in_place,
                        double* x_ref,
                        float r_list, unsigned* d_err, const unsigned* d_gate, cudaStream_t st)
{
    const int T = 256;
    const float rv2 = r_list * r_list;
    const bool cells = b.nc[0] > 0;
    const int ncell = cells ? b.nc[0] * b.nc[1] * b.nc[2] : 0;
    k_bin<<<blocks_for(n, T), T, 0, st>>>(n, pos, zatom, wrap_in_place ? 1 : 0, x_ref, nl.xh, nl.xl, nl.atom_cell,
                                          nl.cell_count, b, d_gate, d_err);
    if (cells) {
        k_scan<<<1, kScanThreads, 0, st>>>(ncell, nl.cell_count, nl.cell_start, nl.cell_fill, d_gate);
        k_scatter<<<blocks_for(n, T), T, 0, st>>>(n, nl.atom_cell, nl.cell_start, nl.cell_fill, nl.cell_atoms,
                                                  d_gate);
        // per-warp list buffer: a power of two >= m_cap entries of (key, value)
        int lcap = 32;
        while (lcap < nl.m_cap) lcap <<= 1;
        const size_t smem = (size_t)kVerletWarps * (3 * lcap + kVerletCellWords) * sizeof(float);
        k_verlet_cells<<<std::min(blocks_for(n, kVerletWarps), kListGridCap), 32 * kVerletWarps, smem, st>>>(
            n, nl.m_cap, lcap, rv2, nl.xh, nl.xl, nl.atom_cell, nl.cell_start, nl.cell_atoms, nl.count, nl.nbr, nl.pf,
            nl.vala, d_err, b, d_gate);
    } else {
        k_verlet_brute<<<blocks_for(n, 128), 128, 0, st>>>(n, nl.m_cap, rv2, nl.xh, nl.xl, nl.count, nl.nbr, nl.pf,
                                                           nl.vala, d_err, b, d_gate);
    }
    k_reverse<<<std::min(blocks_for(n, 4), kListGridCap), 128, 0, st>>>(n, nl.m_cap, nl.count, nl.pf, nl.vala, nl.rev,
                                                                         d_err, d_gate);
    return cuda_fail(cudaGetLastError(), "neighbour-list kernels");
}

}  // namespace nep
