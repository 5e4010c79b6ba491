// Host-side preprocessing of libfem (Section 3 set-up, Section 4 data
// structures): element geometry and conductances, reverse Cuthill-McKee,
// block partition, node classification, shared-memory schedules.
// Pure C++ (no CUDA).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "fem_internal.h"

namespace fem {

// node -> incident elements (CSR)
struct NodeElems {
    std::vector<int64_t> ptr;   // [N+1]
    std::vector<int32_t> elem;  // [4E]
};
void build_node_elems(int64_t N, int64_t E, const int32_t *tets, NodeElems &out);

// Signed volume and the six off-diagonal conductances w_ab = -K^e_ab,
// pairs (0,1) (0,2) (0,3) (1,2) (1,3) (2,3), of one tet (Eq. 9).  The
// shape-function gradients are formed from the face area vectors: grad N_a
// is the inward area vector of the face opposite corner a divided by 3|V|.
double tet_signed_volume(const double *x0, const double *x1, const double *x2,
                         const double *x3);
void tet_conductances(const double *x0, const double *x1, const double *x2,
                      const double *x3, double k, double w[6], double *abs_vol);

// Max |i - j| over node pairs of an element; perm may be null (identity).
int64_t mesh_bandwidth(int64_t E, const int32_t *tets, const int32_t *perm);

// Reverse Cuthill-McKee: perm[old] = new.
void rcm_order(int64_t N, int64_t E, const int32_t *tets, const NodeElems &adj,
               std::vector<int32_t> &perm);

// Face ownership: for each face the unique tet having it as a face, or an
// error message naming the first face that is not a face of exactly one tet.
std::string face_owners(int64_t F, const int32_t *faces, const int32_t *tets,
                        const NodeElems &adj, std::vector<int32_t> &owner);

// Greedy element colouring (no two elements of one colour share a node),
// visiting elements in the given order.  Returns the number of colours.
int greedy_color(int64_t N, int64_t E, const int32_t *tets, const int32_t *order,
                 std::vector<int32_t> &color);

// Block-variant plan.
struct BlockPlan {
    int64_t N = 0, E = 0, F = 0;
    int64_t n_int = 0, n_sh = 0, n_copies = 0, n_rounds = 0, n_sched_words = 0;
    int64_t chunk_stride = 0;         // 32-bit words between blocks' schedule chunks
    int64_t E_pad = 0, F_pad = 0;
    int32_t max_ne = 0;
    size_t max_slots = 0, max_nloc = 0;
    std::vector<BlockInfo> blocks;
    std::vector<int32_t> node_new;    // caller -> internal
    std::vector<int32_t> node_old;    // internal -> caller
    std::vector<int32_t> elem_order;  // [E_pad] caller element or -1
    std::vector<int32_t> face_order;  // [F_pad] caller face or -1
    std::vector<int32_t> copy_node;   // [n_copies]
    std::vector<int32_t> sh_ptr;      // [n_sh+1]
    std::vector<int32_t> sh_copy;     // [n_copies] copy index of each (node, block)
    std::vector<int32_t> copy_pos;    // [n_copies] position of a copy's partial in the
                                      // node-ordered partial array (inverse of sh_copy)
    std::vector<int32_t> grp;         // group -> first round (per block ngrp+1)
    std::vector<uint16_t> sched;      // [n_rounds * 32], pairs of rounds per lane:
                                      // (round r, lane) at (r/2)*64 + 2*lane + r%2
    std::vector<int32_t> elem_nodes;  // [E_pad][4] internal ids (-1 pad)
    std::vector<int32_t> face_nodes;  // [F_pad][3]
    // independent instances (a batch): blocks never mix instances; plan
    // position k holds caller instance inst_order[k], whose blocks are
    // [inst_block_start[k], inst_block_start[k+1]); its interior nodes and
    // its shared nodes are contiguous too (inst_int_start, inst_sh_start)
    std::vector<int32_t> inst_order;
    std::vector<int32_t> inst_block_start;
    std::vector<int64_t> inst_int_start, inst_sh_start;
    std::vector<int32_t> block_inst;  // [n_blocks] caller instance of each block
};

// rank[n]: priority of node n (its position in the chosen node order);
// used to order nodes inside blocks.  face_owner[f]: owning element.
// inst_elem_start: element ranges of independent instances ([n_inst+1],
// empty = one instance); inst_order: plan order of the instances (empty =
// caller order).  Instances must not share nodes.
std::string build_block_plan(int64_t N, int64_t E, const double *xyz, const int32_t *tets,
                             const std::vector<int32_t> &rank, int64_t F,
                             const int32_t *faces, const std::vector<int32_t> &face_owner,
                             int block_elems, int real_size, BlockPlan &out,
                             const std::vector<int64_t> &inst_elem_start = {},
                             const std::vector<int32_t> &inst_order = {});

// Bank-aware order of the slots inside every 32-lane group of the schedule
// (called by build_block_plan; real_size 4 or 8 selects the bank model).
void bank_schedule(BlockPlan &bp, int real_size);

// Flat (atomic / coloured) plan: nodes in rank order, elements sorted by
// (colour, smallest internal node).
struct FlatPlan {
    int64_t N = 0, E = 0, F = 0, E_pad = 0, F_pad = 0;
    std::vector<int32_t> node_new, node_old;
    std::vector<int32_t> elem_order;   // [E_pad] caller element or -1
    std::vector<int32_t> face_order;   // [F_pad]
    std::vector<int64_t> color_start;  // [n_colors+1] element positions (coloured)
    int n_colors = 0;
};
std::string build_flat_plan(int64_t N, int64_t E, const int32_t *tets,
                            const std::vector<int32_t> &rank, int64_t F, bool colored,
                            FlatPlan &out);

// Gershgorin stable step (reading of Eq. 13): 2 / max_i sum_j |(K+H)_ij| / C_i.
// w: [E][6] conductances in the caller's corner order; fa: [F] h A/12.  The
// last F_if faces are interface faces (Eq. 8) whose ambient temperature is
// the mean of the sister face's nodes sister_nodes[F_if][3].
double gershgorin_dt(int64_t N, int64_t E, const int32_t *tets, const double *w,
                     const NodeElems &adj, int64_t F, const int32_t *faces,
                     const double *fa, const double *C, const uint8_t *is_dir,
                     int64_t F_if = 0, const int32_t *sister_nodes = nullptr);

// Sister of every interface face (Eq. 8, Section 3): faces [n_a + n_b][3]
// (side A first), the index of the other side's face with the nearest
// centroid, ties to the lower index.
void interface_sisters(const double *xyz, int64_t n_a, int64_t n_b, const int32_t *faces,
                       std::vector<int64_t> &sister);

}  // namespace fem
