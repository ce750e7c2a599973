// nep_neighbor.cu -- cell binning and Verlet neighbour list on the device.
//
// The paper keeps neighbour lists of atoms within the cutoffs (Sec. III.C,
// "memory consumption") without describing their construction.  Here:
//   1. wrap positions into the orthorhombic box, split them into FP32 hi/lo,
//      bin atoms into cells of edge >= the list radius;
//   2. exclusive scan of the cell counts and scatter (the order of atoms
//      within a cell is whatever the atomics give: the list order below
//      depends only on the sort keys, so it stays deterministic);
//   3. every pair within the list radius is tested once, by the atom whose
//      half shell of cells holds the other, and goes into both atoms' rows
//      (full list, both directions), unsorted; each row is then ordered by
//      increasing distance, and the reverse-pair index (for slot k of atom
//      i, the slot of i in j's list) follows from the partners' ranks
//      (k_half_cells, k_sort_tile, k_rev_tile below);
// Boxes with fewer than 3 cells in a direction (small training cells) use a
// brute-force scan over all atoms and images, the rows sorted in place
// (keys atom-major in the partial-force buffer, the values in vala), and
// the reverse index by binary search over j's keys (k_reverse).
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
                      int* __restrict__ atom_cell, int* __restrict__ cell_count, int* __restrict__ count, Box b,
                      const unsigned* gate, unsigned* __restrict__ err)
{
    if (gated_off(gate)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    count[i] = 0;  // the half-shell search counts each row's entries with atomics
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

// Warps per block of the warp-per-atom list kernels.
constexpr int kVerletWarps = 4;

// (squared distance, packed index) as one unsigned 64-bit sort key: d2 >= 0,
// so its IEEE bits order like its value, and the packed index is below 2^31.
__device__ __forceinline__ unsigned long long sort_key(float d2, int v)
{
    return ((unsigned long long)__float_as_uint(d2) << 32) | (unsigned)v;
}

// The list in three steps, each pair's distance tested once (the cells path):
//   k_half_cells  one warp per atom i scans the 14 cells of its half shell
//                 (cell offsets after (0, 0, 0) in x-slowest order, and its
//                 own cell for j > i), so that every pair within the list
//                 radius is met by exactly one of its two atoms; the
//                 quick hi-part test and the exact hi/lo test as before, and
//                 each accepted pair goes into both rows unsorted at slots
//                 taken with atomics: (value, distance word, the partner
//                 entry's slot).  The rows live in the partial-force buffer,
//                 four words per slot.
//   k_sort_tile   one warp per atom ranks its row by (squared distance,
//                 value), which is unique, and writes the sorted values
//                 (slot-major nbr, through a shared tile of 32 atoms so that
//                 the stores are whole rows), the rank of every unsorted
//                 slot (vala), and into the fourth word of each partner
//                 entry the rank it got here: the partner's reverse index
//                 (k_sort_rows, a warp per atom storing nbr directly, above
//                 128 slots).
//   k_rev_tile    rev[rank of slot s][i] = the fourth word of i's slot s,
//                 within each row, 32 atoms per block transposed through
//                 shared memory into whole-row stores (k_rev_perm, a warp
//                 per atom, above 352 slots).
// The pair vector is computed once per pair in the canonical orientation, so
// the rows and the reverse index are the same as those of the full-shell
// search (the order of the unsorted slots, which the atomics decide, does
// not reach the results).  The counts are cleared by k_bin.
constexpr int kHalfCells = 14;

__global__ void __launch_bounds__(32 * kVerletWarps) k_half_cells(int n, int m_cap, float rv2,
                                                                 const float* __restrict__ xh,
                                                                 const float* __restrict__ xl,
                                                                 const int* __restrict__ atom_cell,
                                                                 const int* __restrict__ cell_start,
                                                                 const int* __restrict__ cell_atoms,
                                                                 int* __restrict__ count, int* __restrict__ rows,
                                                                 int lcap, unsigned* err, Box b, const unsigned* gate)
{
    if (gated_off(gate)) return;
    extern __shared__ int s_half[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // per warp: lcap quick-test survivors, 15 prefix sums, 14 starts, codes, shifts
    int* sq = s_half + (size_t)warp * (lcap + 6 * 32);
    int* pre = sq + lcap;
    int* cst = pre + 32;
    int* ccode = cst + 32;
    float* csh = reinterpret_cast<float*>(ccode + 32);
    const float rq = sqrtf(rv2) + 1e-3f, rq2 = rq * rq;
    for (int i = blockIdx.x * kVerletWarps + warp; i < n; i += gridDim.x * kVerletWarps) {
        float hi[3], li[3];
        load_pos(xh, xl, n, i, hi, li);
        const int cid = atom_cell[i];
        const int cz = cid % b.nc[2];
        const int cy = (cid / b.nc[2]) % b.nc[1];
        const int cx = cid / (b.nc[2] * b.nc[1]);
        // lane c < 14 describes half-shell cell c: offset index 13 + c of the
        // 27 in x-slowest order (13 is the atom's own cell)
        int ccount = 0;
        if (lane < kHalfCells) {
            const int o = 13 + lane;
            int x2 = cx + o / 9 - 1, y2 = cy + (o / 3) % 3 - 1, z2 = cz + o % 3 - 1;
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
        int incl = ccount;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane <= kHalfCells) pre[lane] = incl - ccount;
        if (lane < kHalfCells) cst[lane] -= incl - ccount;
        __syncwarp();
        const int total = pre[kHalfCells];
        // pass 1, quick rejection with the hi parts only: their pair vector is
        // within 1e-4 A of the hi/lo one, so the 1e-3 A margin never drops a
        // pair that the exact test keeps; survivors are compacted into sq
        int nq = 0, c0 = 0;
        for (int base = 0; base < total; base += 32) {
            const int idx = base + lane;
            bool pass = false;
            int value = 0;
            int c = c0;
            if (idx < total) {
                while (pre[c + 1] <= idx) ++c;
                const int j = cell_atoms[cst[c] + idx];
                // own cell (c == 0): the pairs with j > i only
                if (c != 0 || j > i) {
                    const float4 a = NEP_LDG(reinterpret_cast<const float4*>(xh) + j);
                    const float qx = (a.x - hi[0]) + csh[c];
                    const float qy = (a.y - hi[1]) + csh[32 + c];
                    const float qz = (a.z - hi[2]) + csh[64 + c];
                    pass = j != i && fmaf(qx, qx, fmaf(qy, qy, qz * qz)) < rq2;
                    value = j | (ccode[c] << 24);
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
        // pass 2: the exact test; an accepted pair takes a slot in i's row
        // (one atomic per warp round) and one in j's row
        const int nqs = nq < lcap ? nq : lcap;
        for (int base = 0; base < nqs; base += 32) {
            const int e = base + lane;
            bool accept = false;
            int value = 0, j = 0;
            float d2 = 0.f;
            if (e < nqs) {
                value = sq[e];
                j = value & 0xFFFFFF;
                float hj[3], lj[3];
                load_pos(xh, xl, n, j, hj, lj);
                float rx, ry, rz;
                pair_vector(i, j, value >> 24, hi, li, hj, lj, b, rx, ry, rz);
                d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                accept = d2 < rv2;
            }
            const unsigned mask = __ballot_sync(0xffffffffu, accept);
            int si0 = 0;
            if (lane == 0 && mask) si0 = atomicAdd(count + i, __popc(mask));
            si0 = __shfl_sync(0xffffffffu, si0, 0);
            if (accept) {
                const int si = si0 + __popc(mask & ((1u << lane) - 1u));
                const int sj = atomicAdd(count + j, 1);
                const int vj = i | ((124 - (value >> 24)) << 24);  // the reverse image
                if (si < m_cap) {
                    int* ri = rows + ((size_t)i * m_cap + si) * 4;
                    ri[0] = value;
                    ri[1] = (int)__float_as_uint(d2);
                    ri[2] = sj;
                }
                if (sj < m_cap) {
                    int* rj = rows + ((size_t)j * m_cap + sj) * 4;
                    rj[0] = vj;
                    rj[1] = (int)__float_as_uint(d2);
                    rj[2] = si;
                }
            }
        }
        __syncwarp();  // the warp's buffers are reused by its next atom
    }
}

// Ranks a warp's row entries c0 + lane + 32 t against all ns (keys in sk)
// and writes each at its rank: the value to out[rank * out_stride] (the
// atom's column of the slot-major nbr, or of a shared-memory tile), the rank
// to inv[i][unsorted slot] and to the fourth word of the partner entry (the
// partner's reverse index; j's slot sp[e] of the atom in the value).
template <int EPL>
__device__ __forceinline__ void rank_rows_write(int c0, int ns, int m, int lane, const unsigned long long* sk,
                                                const int* sp, int i, int out_stride, int m_cap, int* out,
                                                int* __restrict__ rows, int* __restrict__ inv)
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
        if (e < ns) {
            const int v = (int)(unsigned)ke[t];
            inv[(size_t)i * m_cap + e] = rk[t];
            out[(size_t)rk[t] * out_stride] = v;
            const int ps = sp[e];
            if (ps < m_cap) rows[((size_t)(v & 0xFFFFFF) * m_cap + ps) * 4 + 3] = rk[t];
        }
    }
}

__global__ void __launch_bounds__(32 * kVerletWarps) k_sort_rows(int n, int m_cap, int lcap, int* __restrict__ rows,
                                                                const int* __restrict__ count, int* __restrict__ nbr,
                                                                int* __restrict__ inv, unsigned* err,
                                                                const unsigned* gate)
{
    if (gated_off(gate)) return;
    extern __shared__ unsigned long long s_sort[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned long long* sk = s_sort + (size_t)warp * lcap * 3 / 2;  // lcap keys, then lcap partner slots
    int* sp = reinterpret_cast<int*>(sk + lcap);
    // a lane's entries of the next atom's row (e = lane + 32 t), loaded while
    // the current row is sorted
    constexpr int kPre = 4;  // 128 entries per row at most
    int4 pre[kPre];
    int pre_cnt = 0;
    const int stride = gridDim.x * kVerletWarps;
    auto fetch = [&](int a) {
        pre_cnt = a < n ? count[a] : 0;
        const int ns_a = min(min(pre_cnt, m_cap), lcap);
#pragma unroll
        for (int t = 0; t < kPre; ++t) {
            const int e = lane + 32 * t;
            if (e < ns_a) pre[t] = *reinterpret_cast<const int4*>(rows + ((size_t)a * m_cap + e) * 4);
        }
    };
    fetch(blockIdx.x * kVerletWarps + warp);
    for (int i = blockIdx.x * kVerletWarps + warp; i < n; i += stride) {
        const int cnt = pre_cnt;
        if (cnt > m_cap && lane == 0) atomicOr(err, kErrOverflow);
        const int m = cnt < m_cap ? cnt : m_cap;
        const int ns = m < lcap ? m : lcap;
#pragma unroll
        for (int t = 0; t < kPre; ++t) {
            const int e = lane + 32 * t;
            if (e < ns) {
                sk[e] = sort_key(__int_as_float(pre[t].y), pre[t].x);
                sp[e] = pre[t].z;
            }
        }
        for (int e = 32 * kPre + lane; e < ns; e += 32) {  // rows longer than the prefetch (m_cap > 128)
            const int4 r = *reinterpret_cast<const int4*>(rows + ((size_t)i * m_cap + e) * 4);
            sk[e] = sort_key(__int_as_float(r.y), r.x);
            sp[e] = r.z;
        }
        __syncwarp();
        fetch(i + stride);
        if (ns <= 32)
            rank_rows_write<1>(0, ns, m, lane, sk, sp, i, n, m_cap, nbr + i, rows, inv);
        else if (ns <= 64)
            rank_rows_write<2>(0, ns, m, lane, sk, sp, i, n, m_cap, nbr + i, rows, inv);
        else
            for (int c0 = 0; c0 < ns; c0 += 128)
                rank_rows_write<4>(c0, ns, m, lane, sk, sp, i, n, m_cap, nbr + i, rows, inv);
        __syncwarp();
    }
}

// The same sort with the slot-major nbr stores made whole: a block of
// kSortWarps warps takes tiles of 32 consecutive atoms in turn, warp w the
// atoms w, w + 8, w + 16, w + 24 of each (the next one's row loaded into
// registers while the current one sorts); the sorted values go to a shared
// tile (atom a's column), stored after the block barrier as rows of 32
// consecutive atoms (one 128-byte store each).  inv and the partner words are
// written as in k_sort_rows.  Shared memory: the warps' key buffers (lcap x
// 12 bytes each), then the m_cap x 33-int tile.
constexpr int kSortWarps = 8;
constexpr int kSortAtoms = 32;
constexpr int kSortGridCap = 152 * 8;
constexpr size_t kSortTileMaxSmem = 48 * 1024;  // up to 128 slots per atom (the warp-per-atom sort beyond)

__global__ void __launch_bounds__(32 * kSortWarps) k_sort_tile(int n, int m_cap, int lcap, int* __restrict__ rows,
                                                              const int* __restrict__ count, int* __restrict__ nbr,
                                                              int* __restrict__ inv, unsigned* err,
                                                              const unsigned* gate)
{
    if (gated_off(gate)) return;
    extern __shared__ unsigned long long s_sort[];
    __shared__ int s_cnt[kSortAtoms];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned long long* sk = s_sort + (size_t)warp * lcap * 3 / 2;  // lcap keys, then lcap partner slots
    int* sp = reinterpret_cast<int*>(sk + lcap);
    int* s_tile = reinterpret_cast<int*>(s_sort + (size_t)kSortWarps * lcap * 3 / 2);  // [m_cap][33]
    constexpr int kPer = kSortAtoms / kSortWarps;  // atoms per warp and tile
    const int tiles = (n + kSortAtoms - 1) / kSortAtoms;
    // this warp's k-th atom: tile blockIdx.x + (k / kPer) gridDim.x, column warp + kSortWarps (k % kPer)
    auto atom_of = [&](int k, int& tile, int& a) {
        tile = blockIdx.x + (k / kPer) * gridDim.x;
        a = warp + kSortWarps * (k % kPer);
        return tile * kSortAtoms + a;
    };
    constexpr int kPre = 4;  // 128 entries per row at most
    int4 pre[kPre];
    int pre_cnt = 0;
    auto fetch = [&](int k) {
        int tile, a;
        const int at = atom_of(k, tile, a);
        pre_cnt = tile < tiles && at < n ? count[at] : 0;
        const int ns_a = min(min(pre_cnt, m_cap), lcap);
#pragma unroll
        for (int t = 0; t < kPre; ++t) {
            const int e = lane + 32 * t;
            if (e < ns_a) pre[t] = *reinterpret_cast<const int4*>(rows + ((size_t)at * m_cap + e) * 4);
        }
    };
    fetch(0);
    for (int k = 0;; ++k) {
        int tile, a;
        const int i = atom_of(k, tile, a);
        if (tile >= tiles) break;
        const int cnt = pre_cnt;  // 0 past the last atom
        if (cnt > m_cap && lane == 0) atomicOr(err, kErrOverflow);
        const int m = cnt < m_cap ? cnt : m_cap;
        const int ns = m < lcap ? m : lcap;
        if (lane == 0) s_cnt[a] = ns;
#pragma unroll
        for (int t = 0; t < kPre; ++t) {
            const int e = lane + 32 * t;
            if (e < ns) {
                sk[e] = sort_key(__int_as_float(pre[t].y), pre[t].x);
                sp[e] = pre[t].z;
            }
        }
        for (int e = 32 * kPre + lane; e < ns; e += 32) {  // rows longer than the prefetch (m_cap > 128)
            const int4 r = *reinterpret_cast<const int4*>(rows + ((size_t)i * m_cap + e) * 4);
            sk[e] = sort_key(__int_as_float(r.y), r.x);
            sp[e] = r.z;
        }
        __syncwarp();
        fetch(k + 1);
        int* col = s_tile + a;
        if (ns == 0) {
        } else if (ns <= 32)
            rank_rows_write<1>(0, ns, m, lane, sk, sp, i, kSortAtoms + 1, m_cap, col, rows, inv);
        else if (ns <= 64)
            rank_rows_write<2>(0, ns, m, lane, sk, sp, i, kSortAtoms + 1, m_cap, col, rows, inv);
        else
            for (int c0 = 0; c0 < ns; c0 += 128)
                rank_rows_write<4>(c0, ns, m, lane, sk, sp, i, kSortAtoms + 1, m_cap, col, rows, inv);
        __syncwarp();
        if (k % kPer == kPer - 1) {
            // the tile is complete: its rows to nbr, 32 consecutive atoms each
            __syncthreads();
            const int i0 = tile * kSortAtoms;
            const int ca = s_cnt[lane];
            for (int r = warp; r < m_cap; r += kSortWarps)
                if (r < ca) nbr[(size_t)r * n + i0 + lane] = s_tile[r * (kSortAtoms + 1) + lane];
            __syncthreads();  // the tile and the counts are read before the next tile writes them
        }
    }
}

// rev[inv[i][s]][i] = the reverse index left in the fourth word of i's
// unsorted slot s by the partner's sort; one warp per atom.  A value outside
// the partner's kept entries (only after an overflow, already latched) is
// latched again and replaced by the slot's own rank.
__global__ void k_rev_perm(int n, int m_cap, const int* __restrict__ count, const int* __restrict__ rows,
                           const int* __restrict__ inv, int* __restrict__ rev, unsigned* err, const unsigned* gate)
{
    if (gated_off(gate)) return;
    const int lane = threadIdx.x & 31;
    const int warps = (int)((gridDim.x * blockDim.x) >> 5);
    for (int i = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); i < n; i += warps) {
        const int ci = min(count[i], m_cap);
        for (int s = lane; s < ci; s += 32) {
            const int r = inv[(size_t)i * m_cap + s];
            int v = rows[((size_t)i * m_cap + s) * 4 + 3];
            if (v < 0 || v >= m_cap) {
                atomicOr(err, kErrReverse);
                v = r;
            }
            rev[(size_t)r * n + i] = v;
        }
    }
}

// The same reverse index with the slot-major stores made whole: a block of
// eight warps takes tiles of 32 consecutive atoms in turn; each warp fills the shared tile
// columns of its atoms (rev value of sorted slot r of atom a at tile[r][a],
// reading the rows as k_rev_perm does), then each warp stores tile rows, 32
// consecutive atoms per 128-byte store.  Slots at or past an atom's count are
// not stored.  Shared memory: m_cap x 33 ints.
constexpr int kRevAtoms = 32;
constexpr int kRevThreads = 256;
constexpr int kRevTileMaxSlots = 352;  // 352 x 33 x 4 bytes stay under 48 KB
constexpr int kRevGridCap = 152 * 8;   // blocks walk the 32-atom tiles; a gated-off launch retires fast

__global__ void __launch_bounds__(kRevThreads) k_rev_tile(int n, int m_cap, const int* __restrict__ count,
                                                          const int* __restrict__ rows, const int* __restrict__ inv,
                                                          int* __restrict__ rev, unsigned* err, const unsigned* gate)
{
    if (gated_off(gate)) return;
    extern __shared__ int s_tile[];  // [m_cap][kRevAtoms + 1]
    __shared__ int s_cnt[kRevAtoms];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles = (n + kRevAtoms - 1) / kRevAtoms;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int i0 = tile * kRevAtoms;
        if (threadIdx.x < kRevAtoms) {
            const int i = i0 + threadIdx.x;
            s_cnt[threadIdx.x] = i < n ? min(count[i], m_cap) : 0;
        }
        __syncthreads();
        for (int a = warp; a < kRevAtoms; a += kRevThreads / 32) {
            const int i = i0 + a, ci = s_cnt[a];
            for (int s = lane; s < ci; s += 32) {
                const int r = inv[(size_t)i * m_cap + s];
                int v = rows[((size_t)i * m_cap + s) * 4 + 3];
                if (v < 0 || v >= m_cap) {
                    atomicOr(err, kErrReverse);
                    v = r;
                }
                if (r >= 0 && r < ci)
                    s_tile[r * (kRevAtoms + 1) + a] = v;
                else
                    atomicOr(err, kErrReverse);
            }
        }
        __syncthreads();
        const int ca = s_cnt[lane];
        for (int r = warp; r < m_cap; r += kRevThreads / 32)
            if (r < ca) rev[(size_t)r * n + i0 + lane] = s_tile[r * (kRevAtoms + 1) + lane];
        __syncthreads();  // the tile and the counts are read before the next tile writes them
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
                                          nl.cell_count, nl.count, b, d_gate, d_err);
    if (cells) {
        k_scan<<<1, kScanThreads, 0, st>>>(ncell, nl.cell_count, nl.cell_start, nl.cell_fill, d_gate);
        k_scatter<<<blocks_for(n, T), T, 0, st>>>(n, nl.atom_cell, nl.cell_start, nl.cell_fill, nl.cell_atoms,
                                                  d_gate);
        // per-warp buffers: a power of two >= m_cap entries
        int lcap = 32;
        while (lcap < nl.m_cap) lcap <<= 1;
        const int grid = std::min(blocks_for(n, kVerletWarps), kListGridCap);
        int* rows = reinterpret_cast<int*>(nl.pf);  // four words per slot, free until the site pass
        k_half_cells<<<grid, 32 * kVerletWarps, (size_t)kVerletWarps * (lcap + 6 * 32) * sizeof(int), st>>>(
            n, nl.m_cap, rv2, nl.xh, nl.xl, nl.atom_cell, nl.cell_start, nl.cell_atoms, nl.count, rows, lcap, d_err, b,
            d_gate);
        const size_t sort_smem = (size_t)kSortWarps * lcap * 12 + (size_t)nl.m_cap * (kSortAtoms + 1) * sizeof(int);
        if (sort_smem <= kSortTileMaxSmem)
            k_sort_tile<<<std::min(blocks_for(n, kSortAtoms), kSortGridCap), 32 * kSortWarps, sort_smem, st>>>(
                n, nl.m_cap, lcap, rows, nl.count, nl.nbr, nl.vala, d_err, d_gate);
        else
            k_sort_rows<<<grid, 32 * kVerletWarps, (size_t)kVerletWarps * lcap * 12, st>>>(
                n, nl.m_cap, lcap, rows, nl.count, nl.nbr, nl.vala, d_err, d_gate);
        if (nl.m_cap <= kRevTileMaxSlots)
            k_rev_tile<<<std::min(blocks_for(n, kRevAtoms), kRevGridCap), kRevThreads,
                         (size_t)nl.m_cap * (kRevAtoms + 1) * sizeof(int), st>>>(n, nl.m_cap, nl.count, rows,
                                                                                  nl.vala, nl.rev, d_err, d_gate);
        else
            k_rev_perm<<<std::min(blocks_for(n, 4), kListGridCap), 128, 0, st>>>(n, nl.m_cap, nl.count, rows,
                                                                                  nl.vala, nl.rev, d_err, d_gate);
        return cuda_fail(cudaGetLastError(), "neighbour-list kernels");
    } else {
        k_verlet_brute<<<blocks_for(n, 128), 128, 0, st>>>(n, nl.m_cap, rv2, nl.xh, nl.xl, nl.count, nl.nbr, nl.pf,
                                                           nl.vala, d_err, b, d_gate);
    }
    k_reverse<<<std::min(blocks_for(n, 4), kListGridCap), 128, 0, st>>>(n, nl.m_cap, nl.count, nl.pf, nl.vala, nl.rev,
                                                                         d_err, d_gate);
    return cuda_fail(cudaGetLastError(), "neighbour-list kernels");
}

}  // namespace nep
