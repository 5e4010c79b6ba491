// What the learned surrogate (fem_surrogate.cu) reads from and writes to a
// mesh (implemented in fem_api.cpp).  Not part of the ABI.
#pragma once

#include <cstdint>

#include "fem_internal.h"

struct fem_mesh;

namespace fem {

// What the learned surrogate (fem_surrogate.cu) reads from a mesh: host data
// in the caller's order and the plan's node numbering (fem_api.cpp).
struct SurrogateMeshView {
    int64_t N, E;
    const double *xyz;          // [N][3]
    const int32_t *tets;        // [E][4]
    const double *w;            // [E][6] w_ab = -K^e_ab, pairs (0,1) (0,2) (0,3) (1,2) (1,3) (2,3)
    const double *C, *Lc;       // lumped capacities [N]
    const uint8_t *rng_id;      // phase-change range index [N]
    const double *ranges;       // [n_ranges][2] (Ts, Tl)
    int32_t n_ranges;
    int64_t F_rb;               // Robin faces
    const int32_t *rb_faces;    // [F_rb][3]
    const double *rb_fa, *rb_fg;  // h A / 12, A/3 (h T_inf - q)
    int32_t n_inst;             // batch instances (0: a plain mesh)
    const int64_t *inst_node;   // [n_inst + 1]
    const double *inst_dt;      // [n_inst] current per-instance steps
    int32_t prec, variant, formulation;
    int32_t has_kt, has_dir;
    int64_t F_if;
    const int32_t *node_new;    // caller node -> internal node of the block plan
};
// Host view (builds the plan if needed).  Errors as the fem_* calls.
int surrogate_mesh_view(struct ::fem_mesh *m, SurrogateMeshView *v);
// The device state of an FP32 block-variant mesh (uploads it if needed):
// where E of internal node i lives, the mesh's stream and device.
int surrogate_mesh_device(struct ::fem_mesh *m, StateView<float> *v, void **stream, int *device);
// After the surrogate wrote E through the view: refresh the shared-node
// mirrors and advance the step count and time by n_steps steps (each
// instance of a batch by its own step; a plain mesh by dt); the energy
// account no longer balances (the boundary heat of those steps is not
// accumulated).
int surrogate_mesh_advanced(struct ::fem_mesh *m, int64_t n_steps, double dt);

}  // namespace fem
