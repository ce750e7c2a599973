// nep_neighbor.cu -- cell binning and Verlet neighbour list on the device.
//
// The paper keeps neighbour lists of atoms within the cutoffs (Sec. III.C,
// "memory consumption") without describing their construction.  Here:
//   1. wrap positions into the orthorhombic box, split them into FP32 hi/lo,
//      bin atoms into cells of edge >= the list radius;
//   2. exclusive scan of the cell counts, scatter, then sort each cell by
//      atom index so the list order (hence every FP32 sum) is deterministic;
//   3. one thread per atom scans the 27 neighbouring cells and keeps every
//      (j, image) with |r_ij| below the list radius (full list, both
//      directions), then orders its slots by increasing distance (the
//      partial-force buffer is free at this point and holds the sort keys);
//   4. the reverse-pair index: for slot k of atom i, the slot of i in j's list.
// Boxes with fewer than 3 cells in a direction (small training cells) use a
// brute-force scan over all atoms and images instead of cells.
// Every kernel takes an optional device gate word: when it is zero the kernel
// returns at once, which lets the MD step skip the rebuild without a host
// round trip.
#include <cstdio>

#include "nep_internal.cuh"

namespace nep {

namespace {

__device__ __forceinline__ bool gated_off(const unsigned* gate)
{
    return gate != nullptr && *((volatile const unsigned*)gate) == 0u;
}

__global__ void k_bin(int n, double* __restrict__ pos, int wrap_in_place, double* __restrict__ x_ref,
                      float* __restrict__ xh, float* __restrict__ xl, int* __restrict__ atom_cell,
                      int* __restrict__ cell_count, Box b, const unsigned* gate)
{
    if (gated_off(gate)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double L = b.L[d];
        double x = pos[(size_t)d * n + i];
        double w = x - L * floor(x / L);
        if (w >= L) w -= L;
        if (w < 0.0) w = 0.0;
        if (wrap_in_place) {
            pos[(size_t)d * n + i] = w;
            if (x_ref) x_ref[(size_t)d * n + i] = w;
        }
        float h, l;
        split_hilo(w, h, l);
        xh[(size_t)d * n + i] = h;
        xl[(size_t)d * n + i] = l;
        if (b.nc[0] > 0) {
            int ci = (int)(w * (double)b.nc[d] / L);
            c[d] = ci < 0 ? 0 : (ci >= b.nc[d] ? b.nc[d] - 1 : ci);
        }
    }
    if (b.nc[0] > 0) {
        const int cid = (c[0] * b.nc[1] + c[1]) * b.nc[2] + c[2];
        atom_cell[i] = cid;
        atomicAdd(cell_count + cid, 1);
    }
}

// Single-block exclusive scan: cell_start[c] = sum_{c' < c} count[c'].
__global__ void k_scan(int ncell, const int* __restrict__ count, int* __restrict__ start, const unsigned* gate)
{
    if (gated_off(gate)) return;
    __shared__ int part[1024];
    const int t = threadIdx.x, T = blockDim.x;
    const int chunk = (ncell + T - 1) / T;
    const int lo = t * chunk, hi = min(ncell, lo + chunk);
    int s = 0;
    for (int c = lo; c < hi; ++c) s += count[c];
    part[t] = s;
    __syncthreads();
    // Hillis-Steele inclusive scan over the chunk sums
    for (int o = 1; o < T; o <<= 1) {
        int v = (t >= o) ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - s;  // exclusive prefix of this chunk
    for (int c = lo; c < hi; ++c) {
        start[c] = run;
        run += count[c];
    }
    if (t == T - 1) start[ncell] = part[T - 1];
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

// Sort each cell's atoms by index (insertion sort; cells hold ~10 atoms),
// and reset the per-cell counters for the next build.
__global__ void k_sort_cells(int ncell, const int* __restrict__ cell_start, int* __restrict__ cell_atoms,
                             int* __restrict__ cell_count, int* __restrict__ cell_fill, const unsigned* gate)
{
    if (gated_off(gate)) return;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int lo = cell_start[c], hi = cell_start[c + 1];
    for (int a = lo + 1; a < hi; ++a) {
        const int key = cell_atoms[a];
        int b = a - 1;
        while (b >= lo && cell_atoms[b] > key) {
            cell_atoms[b + 1] = cell_atoms[b];
            --b;
        }
        cell_atoms[b + 1] = key;
    }
    cell_count[c] = 0;
    cell_fill[c] = 0;
}

__device__ __forceinline__ void list_push(int i, int n, int m_cap, int& cnt, int value, float d2, int* __restrict__ nbr,
                                          float* __restrict__ key)
{
    if (cnt < m_cap) {
        nbr[(size_t)cnt * n + i] = value;
        key[(size_t)cnt * n + i] = d2;
    }
    ++cnt;
}

// Order atom i's slots by increasing distance (insertion sort, stable).  Slot
// k then holds roughly the k-th nearest neighbour of every atom, so the lanes
// of a warp agree on which slots need the (long) angular work, and the force
// pass can add the nearest (largest) terms last by walking ranks downwards.
__device__ void sort_near_first(int i, int n, int cnt, int* __restrict__ nbr, float* __restrict__ key)
{
    for (int a = 1; a < cnt; ++a) {
        const float kd = key[(size_t)a * n + i];
        const int kv = nbr[(size_t)a * n + i];
        int b = a - 1;
        while (b >= 0 && key[(size_t)b * n + i] > kd) {
            key[(size_t)(b + 1) * n + i] = key[(size_t)b * n + i];
            nbr[(size_t)(b + 1) * n + i] = nbr[(size_t)b * n + i];
            --b;
        }
        key[(size_t)(b + 1) * n + i] = kd;
        nbr[(size_t)(b + 1) * n + i] = kv;
    }
}

// One thread per atom.  Each thread keeps its accepted neighbours sorted by
// distance in its own column of shared memory (entry k of thread t at
// k * blockDim + t, so the lanes of a warp never share a bank) and writes the
// sorted list out once.  Ties keep the candidate order (stable insertion).
__global__ void k_verlet_cells(int n, int m_cap, float rv2, const float* __restrict__ xh,
                               const float* __restrict__ xl, const int* __restrict__ atom_cell,
                               const int* __restrict__ cell_start, const int* __restrict__ cell_atoms,
                               int* __restrict__ count, int* __restrict__ nbr, float* __restrict__ key, unsigned* err,
                               Box b, const unsigned* gate)
{
    if (gated_off(gate)) return;
    extern __shared__ float s_list[];
    const int T = blockDim.x, tid = threadIdx.x;
    float* s_key = s_list;
    int* s_val = reinterpret_cast<int*>(s_list + (size_t)m_cap * T);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float hi[3], li[3];
    load_pos(xh, xl, n, i, hi, li);
    const int cid = atom_cell[i];
    const int cz = cid % b.nc[2];
    const int cy = (cid / b.nc[2]) % b.nc[1];
    const int cx = cid / (b.nc[2] * b.nc[1]);
    int cnt = 0;
    for (int ox = -1; ox <= 1; ++ox) {
        int x2 = cx + ox, sx = 0;
        if (x2 < 0) { x2 += b.nc[0]; sx = -1; } else if (x2 >= b.nc[0]) { x2 -= b.nc[0]; sx = 1; }
        for (int oy = -1; oy <= 1; ++oy) {
            int y2 = cy + oy, sy = 0;
            if (y2 < 0) { y2 += b.nc[1]; sy = -1; } else if (y2 >= b.nc[1]) { y2 -= b.nc[1]; sy = 1; }
            for (int oz = -1; oz <= 1; ++oz) {
                int z2 = cz + oz, sz = 0;
                if (z2 < 0) { z2 += b.nc[2]; sz = -1; } else if (z2 >= b.nc[2]) { z2 -= b.nc[2]; sz = 1; }
                const int code = image_code(sx, sy, sz);
                const int c2 = (x2 * b.nc[1] + y2) * b.nc[2] + z2;
                const int e = cell_start[c2 + 1];
                for (int t = cell_start[c2]; t < e; ++t) {
                    const int j = cell_atoms[t];
                    if (j == i && code == kImgCenter) continue;
                    float hj[3], lj[3];
                    load_pos(xh, xl, n, j, hj, lj);
                    float rx, ry, rz;
                    pair_vector(i, j, code, hi, li, hj, lj, b, rx, ry, rz);
                    const float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                    if (d2 < rv2) {
                        if (cnt < m_cap) {
                            int q = cnt - 1;
                            while (q >= 0 && s_key[q * T + tid] > d2) {
                                s_key[(q + 1) * T + tid] = s_key[q * T + tid];
                                s_val[(q + 1) * T + tid] = s_val[q * T + tid];
                                --q;
                            }
                            s_key[(q + 1) * T + tid] = d2;
                            s_val[(q + 1) * T + tid] = j | (code << 24);
                        }
                        ++cnt;
                    }
                }
            }
        }
    }
    count[i] = cnt;
    if (cnt > m_cap) atomicOr(err, kErrOverflow);
    const int m = cnt < m_cap ? cnt : m_cap;
    for (int k = 0; k < m; ++k) {
        nbr[(size_t)k * n + i] = s_val[k * T + tid];
        key[(size_t)k * n + i] = s_key[k * T + tid];
    }
}

__global__ void k_verlet_brute(int n, int m_cap, float rv2, const float* __restrict__ xh,
                               const float* __restrict__ xl, int* __restrict__ count, int* __restrict__ nbr,
                               float* __restrict__ key, unsigned* err, Box b, const unsigned* gate)
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
    sort_near_first(i, n, cnt < m_cap ? cnt : m_cap, nbr, key);
}

// rev[k][i] = slot of (i, -image) in j's list.  The pair vectors are exactly
// antisymmetric, so both directions carry the same squared distance and j's
// list (sorted by it) is binary-searched; a miss (only possible after an
// overflow) is latched as an error.
__global__ void k_reverse(int n, int m_cap, const int* __restrict__ count, const int* __restrict__ nbr,
                          const float* __restrict__ key, int* __restrict__ rev, unsigned* err, const unsigned* gate)
{
    if (gated_off(gate)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int ci = min(count[i], m_cap);
    for (int k = 0; k < ci; ++k) {
        const int v = nbr[(size_t)k * n + i];
        const int j = v & 0xFFFFFF;
        const int target = i | ((124 - (v >> 24)) << 24);
        const float kd = key[(size_t)k * n + i];
        const int cj = min(count[j], m_cap);
        int lo = 0, hi = cj;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (key[(size_t)mid * n + j] < kd)
                lo = mid + 1;
            else
                hi = mid;
        }
        int found = -1;
        for (int t = lo; t < cj && key[(size_t)t * n + j] == kd; ++t)
            if (nbr[(size_t)t * n + j] == target) {
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

inline int blocks_for(int n, int t) { return (n + t - 1) / t; }

}  // namespace

int build_neighbor_list(NeighborList& nl, const Box& b, int n, double* pos, bool wrap_in_place, double* x_ref,
                        float r_list, unsigned* d_err, const unsigned* d_gate, cudaStream_t st)
{
    const int T = 256;
    const float rv2 = r_list * r_list;
    const bool cells = b.nc[0] > 0;
    const int ncell = cells ? b.nc[0] * b.nc[1] * b.nc[2] : 0;
    k_bin<<<blocks_for(n, T), T, 0, st>>>(n, pos, wrap_in_place ? 1 : 0, x_ref, nl.xh, nl.xl, nl.atom_cell,
                                          nl.cell_count, b, d_gate);
    if (cells) {
        k_scan<<<1, 1024, 0, st>>>(ncell, nl.cell_count, nl.cell_start, d_gate);
        k_scatter<<<blocks_for(n, T), T, 0, st>>>(n, nl.atom_cell, nl.cell_start, nl.cell_fill, nl.cell_atoms,
                                                  d_gate);
        k_sort_cells<<<blocks_for(ncell, T), T, 0, st>>>(ncell, nl.cell_start, nl.cell_atoms, nl.cell_count,
                                                         nl.cell_fill, d_gate);
        // per-thread sorted lists in shared memory: m_cap x 8 bytes per thread
        const int TV = 64;
        const size_t smem = (size_t)nl.m_cap * TV * (sizeof(float) + sizeof(int));
        if (smem > 48 * 1024) {
            int rc = cuda_fail(cudaFuncSetAttribute(k_verlet_cells, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    (int)smem),
                               "neighbour-list shared memory");
            if (rc) return rc;
        }
        k_verlet_cells<<<blocks_for(n, TV), TV, smem, st>>>(n, nl.m_cap, rv2, nl.xh, nl.xl, nl.atom_cell,
                                                            nl.cell_start, nl.cell_atoms, nl.count, nl.nbr, nl.pf,
                                                            d_err, b, d_gate);
    } else {
        k_verlet_brute<<<blocks_for(n, 128), 128, 0, st>>>(n, nl.m_cap, rv2, nl.xh, nl.xl, nl.count, nl.nbr, nl.pf,
                                                           d_err, b, d_gate);
    }
    k_reverse<<<blocks_for(n, 128), 128, 0, st>>>(n, nl.m_cap, nl.count, nl.nbr, nl.pf, nl.rev, d_err, d_gate);
    return cuda_fail(cudaGetLastError(), "neighbour-list kernels");
}

}  // namespace nep
