// nep_dataset.cuh -- the device-resident training set shared by the SNES
// evaluation (nep_train.cu) and the force-loss adjoint (nep_adjoint.cu).
//
// Structures of uneven size are concatenated into one set of N atoms, each
// keeping its own orthorhombic periodic box.  Pairs within max(r_c^R, r_c^A)
// are stored in CSR form: the pairs of atom i are p in [pstart[i], pstart[i+1]),
// pj[p] = j | image_code << 24, rev[p] = the slot of the pair (j -> i).
#pragma once

#include <vector>

#include "nep_site.cuh"

namespace nep {

// Jacobian record of one pair, stored at the owner's slot (slot p of atom i
// pointing to j): the radial part of d q_i / d r_ij; the angular 24 x 3 block
// is ang[aidx[p]].
struct PairRec {
    float r[3];   // r_ij of the owning atom i (the vector from i to j)
    float gd[8];  // g_n'(|r|) / |r|, radial orders n = 0..7 (0 beyond r_c^R)
    float pad;
};

// Scratch of the force-loss adjoint.
struct AdjointScratch {
    int n_blocks = 0;          // per-atom kernel blocks the partial buffers hold
    float* pf = nullptr;       // [n_pairs][3] dU_i/dr_ij of the last forward
    float* res = nullptr;      // [N] float4: F_i - F_tar_i of the last forward
    float* z = nullptr;        // [n_par] parameters of the last forward
    double* part = nullptr;    // [n_blocks][n_par] per-block FP64 partial sums
    double* sums = nullptr;    // [2]: sum |F - F_tar|^2, L_f
    bool ready = false;        // a forward has run since the scratch was made
};

// Launch shapes of the population evaluation.  None of them changes a result
// bit: every value keeps its single writer and its summation order.
constexpr int kMaxWaves = 16;
struct EvalShape {
    int waves = 1;          // the contraction runs over up to this many consecutive ranges of
                            // whole structures; pass 2 of range w overlaps pass 1 of range w + 1
    int owner_warps = 4;    // warps per block of the owner pass (4 or 8)
    int discard = 0;        // pass 2 drops the partial-force lines it has read from L2
    int mlp_threads = 256;  // threads per block of the FP32 network (128 or 256)
    int recv_unroll = 4;    // slots in flight per warp in the receiver pass (4, 8 or 12; 16: staged)
    int fused = 0;          // 0: the two contraction passes; 4, 8 or 16: the fused contraction with
                            // this many members per block (one block per structure and member group)
    int owner_tc = 0;       // 1: in BF16 precision the first of the two passes runs on the tensor
                            // cores (FP16 Jacobian rows x FP16 G, FP32 accumulation)
    int pop_pipe = 0;       // 1: in BF16 precision the population network runs as the pipelined
                            // persistent kernel (same bits)
};

}  // namespace nep

struct nep_dataset {
    nep_model* m = nullptr;
    int S = 0, N = 0;
    long long n_pairs = 0, n_ang = 0, bytes = 0;
    int n_chunks = 0;
    nep::Box* boxes = nullptr;
    int* sid = nullptr;
    int* sstart = nullptr;
    int* s_natoms = nullptr;
    double* s_inv_na = nullptr;  // 1 / atoms of each structure
    float* s_vtar = nullptr;     // [S][8]: virial targets, 1 / atoms (FP32), 0
    int typed = 0;               // species numbers given (multicomponent weighting)
    int* s_chunk0 = nullptr;
    int* s_order = nullptr;      // structures by decreasing atom count (fused contraction blocks)
    int amax = 0;                // atoms of the largest structure
    int* chunk_begin = nullptr;
    int* chunk_end = nullptr;
    float* q = nullptr;
    float* xh = nullptr;  // FP32 hi/lo wrapped positions (float4 records), kept for the adjoint
    float* xl = nullptr;
    float* B = nullptr;
    long long* pstart = nullptr;
    int* pj = nullptr;
    long long* rev = nullptr;   // slot of the reverse pair (j -> i) of each pair
    long long* aidx = nullptr;
    long long* astart = nullptr;  // first angular Jacobian block of each atom [N + 1] (owner order)
    nep::PairRec* rec = nullptr;
    float* ang = nullptr;
    double* e_tar = nullptr;
    float* f_tar = nullptr;
    double* w_tar = nullptr;
    // evaluation scratch (grown on demand)
    int pop_cap = 0;
    float* W1t = nullptr;
    float* b1t = nullptr;
    float* w2t = nullptr;
    float* b2t = nullptr;
    float* G = nullptr;
    double* U = nullptr;
    double* partials = nullptr;  // loss records (ChunkRec, 64 B) [chunk][member]
    unsigned char* packed = nullptr;  // tensor-core operand records
    unsigned char* qpack = nullptr;   // descriptors as split-BF16 A tiles (tensor cores)
    float* pbuf = nullptr;            // [n_pairs][3][Pst] partial forces p_kji at the receiver's slot
    float* w6 = nullptr;              // [N][6][Pst] virial contributions of each owner
    float* fown = nullptr;            // [N][3][Pst] own force terms G_i . B_i
    // the tensor-core owner pass: tiles in owner order, their FP16 Jacobian
    // rows and row scales (built with the set), first tile of each owner (host)
    nep::OwnerTile* tiles = nullptr;
    int n_tiles = 0;
    unsigned char* apack = nullptr;
    float* rowscale = nullptr;
    std::vector<int> h_tile0;
    // force-loss adjoint scratch (grown on demand, nep_adjoint.cu)
    nep::AdjointScratch adj;
    // launch shape of the evaluation (nep_dataset_set_shape / nep_dataset_tune)
    nep::EvalShape shape;
    unsigned long long uid = 0;  // unique per dataset: keys captured generation graphs
    int epoch = 0;               // bumped whenever the evaluation scratch is reallocated
    std::vector<int> h_cb, h_ce;         // host copies of the chunk atom ranges
    std::vector<long long> h_cpairs;     // pairs before each chunk (n_chunks + 1)
    std::vector<int> h_schunk0;          // first chunk of each structure (S + 1)
    cudaStream_t aux = nullptr;          // second stream: pass 2 of one range beside pass 1 of the next
    cudaEvent_t ev_wave[nep::kMaxWaves] = {};
    cudaEvent_t ev_join = nullptr;
};

namespace nep {
// frees the adjoint scratch of a dataset (nep_adjoint.cu)
void free_adjoint(AdjointScratch& a);
}  // namespace nep
