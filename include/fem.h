/*
 * fem.h -- C ABI of libfem: the explicit element-by-element (EBE) enthalpy
 * time step for transient heat conduction with phase change on linear
 * tetrahedra, on one NVIDIA GB300 (sm_103a).
 *
 * Method: R. Tavakoli, "Improvement cache efficiency of explicit finite
 * element procedure and its application to parallel casting solidification
 * simulation" (arXiv 1005.3158): heat equation Eq. 1 with initial condition
 * Eq. 2, Dirichlet Eq. 3 and flux/convective boundaries Eq. 4, in the
 * enthalpy form Eq. 5 (H = integral of C dT, Eq. 11), Galerkin linear tets
 * Eq. 9 with row-sum lumped capacity, explicit update Eq. 14 (theta = 0 of
 * Eq. 10) evaluated as sums of element contributions, Eqs. 15-22.
 * Optional: the apparent-heat-capacity formulation (Eqs. 6-7, Lemmon),
 * temperature-dependent conductivity (Eq. 9's K(T)), the cast-mold
 * interface between non-matching meshes (Eq. 8), and batches of independent
 * meshes advanced together with their own time steps.  Around the step:
 * partition autotuning (fem_autotune) and pipelined host I/O
 * (fem_set_state_async, fem_get_temperature_async, fem_sync).
 *
 * Conventions for every call
 *   - All array arguments are HOST pointers unless stated otherwise.  The
 *     library copies what it needs during the call; the caller keeps
 *     ownership of its arrays and may free them when the call returns.
 *     Output arrays are caller-allocated host arrays of the stated size.
 *   - Node and element ids are 0-based.  All node-indexed inputs and outputs
 *     use the CALLER's node order; any internal reordering is invisible.
 *   - Units: SI (m, kg, s, K, J, W).
 *   - Every call returns a fem_status and never aborts the process.  On an
 *     error the object is left unchanged and fem_last_error() returns a
 *     message for the calling thread.
 *   - A fem_mesh is not thread-safe; use one mesh from one thread at a time.
 *   - Device memory belongs to the library, allocated on the current CUDA
 *     device the first time the mesh needs it (with cudaMalloc, or the
 *     caller's allocator, fem_set_allocator) and released by
 *     fem_mesh_destroy.  Work is enqueued on the mesh's stream (the legacy
 *     default stream unless fem_set_stream was called); the fem_get_* calls
 *     synchronise that stream.  fem_step(n) with n >= 32 replays a CUDA
 *     graph of 32 steps, captured once per time-step size.
 */
#ifndef FEM_H
#define FEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fem_mesh fem_mesh; /* opaque; owned by the library until fem_mesh_destroy */

typedef enum {
    FEM_OK = 0,
    FEM_EINVAL = 1,    /* invalid argument or mesh (message says which) */
    FEM_ENOMEM = 2,    /* host or device allocation failed (nothing leaked) */
    FEM_ECUDA = 3,     /* a CUDA runtime call failed, or no usable GPU */
    FEM_ESTATE = 4,    /* call out of order (e.g. fem_step before materials) */
    FEM_EUNSTABLE = 5, /* non-finite temperatures/energy, or an energy balance
                          residual beyond its rounding bound (fem_get_energy):
                          dt above the stable limit */
    FEM_ETIMEOUT = 6   /* a bounded device wait gave up (reported by the next
                          fem_get_* call; the state is then not valid) */
} fem_status;

typedef enum { FEM_FP64 = 0, FEM_FP32 = 1 } fem_precision;

/* Scatter-add strategy of the element results into nodes (Eqs. 19-22).
 *   FEM_VARIANT_BLOCK   -- default.  Elements are partitioned into blocks
 *                          staged in shared memory; each node sums its
 *                          element-corner results in a fixed order (no
 *                          atomics, bit-reproducible); nodes shared between
 *                          blocks exchange partial sums through a second
 *                          kernel (the paper's exchange of calculated
 *                          values between partitions, Eq. 22).
 *   FEM_VARIANT_ATOMIC  -- every element adds its four results into a global
 *                          nodal array with atomic adds (order-dependent
 *                          rounding; for comparison).
 *   FEM_VARIANT_COLORED -- elements are greedily coloured so that no two
 *                          elements of one colour share a node; one launch
 *                          per colour adds with plain read-modify-write
 *                          (deterministic; for comparison). */
typedef enum { FEM_VARIANT_BLOCK = 0, FEM_VARIANT_ATOMIC = 1, FEM_VARIANT_COLORED = 2 } fem_variant;

/* Nonlinear formulation of the phase change.
 * FEM_ENTHALPY: the enthalpy method (Eq. 5), nodal enthalpy content E as
 *   the unknown, T = T(E); conserves energy exactly.
 * FEM_APPARENT_CAPACITY: the paper's apparent heat capacity (Eqs. 6-7) by
 *   Lemmon's method, T as the unknown: every element's apparent specific
 *   heat is |grad H| / |grad T| from its nodal values (dH/dT at the mean
 *   temperature where T is uniform over it), lumped rho V / 4 per node; each
 *   step solves C_app (T^{n+1} - T^n) / dt = F - K T^n.  Energy is conserved
 *   only approximately.  Block variant only; every phase-change material
 *   needs T_liquidus > T_solidus.  The state I/O (fem_get_state /
 *   fem_set_state) still exchanges E = E(T). */
typedef enum { FEM_ENTHALPY = 0, FEM_APPARENT_CAPACITY = 1 } fem_formulation;

/* One material (Section 2): density rho (kg/m^3), specific heat c (J/kgK),
 * conductivity k (W/mK), latent heat (J/kg) released linearly between
 * T_solidus and T_liquidus (K).  latent == 0 means no phase change (the
 * two temperatures are then ignored); T_solidus == T_liquidus is an
 * isothermal phase change. */
typedef struct {
    double rho, c, k, latent, T_solidus, T_liquidus;
} fem_material;

/* Options of fem_mesh_create_ex.  Zero-initialise and set what you need;
 * zero fields take the defaults. */
typedef struct {
    int32_t variant;     /* fem_variant, default FEM_VARIANT_BLOCK */
    int32_t block_elems; /* target elements per shared-memory block, 0 = auto;
                            clamped to [64, 12288].  Auto: 1024 for FP64;
                            for FP32 1792 when the block kernel reads the
                            conductances from L2 (below), else 2048.  With
                            L2 conductances the automatic size shrinks in
                            64-element steps (not below 1024) until the
                            largest block leaves room for four CTAs per SM. */
    int32_t threads;     /* threads per CTA of the block kernel: 0 = auto,
                            or 128, 256, 512 or 1024.  With constant k and
                            the enthalpy formulation, 0 or 256 selects the
                            kernel that reads the six conductances of each
                            element from L2 (bulk-prefetched) instead of
                            staging them in shared memory, at 256 threads.
                            Otherwise auto is the fewest threads whose
                            16-byte element accesses cover the largest
                            block. */
    int32_t formulation; /* fem_formulation, default FEM_ENTHALPY */
    int32_t reserved[4];
} fem_options;

/* Statistics of the execution plan (fem_mesh_info). */
typedef struct {
    int64_t n_nodes, n_tets, n_faces;
    int64_t n_blocks;          /* element blocks (block variant) */
    int64_t n_interior_nodes;  /* nodes owned by exactly one block */
    int64_t n_shared_nodes;    /* nodes touched by two or more blocks */
    int64_t n_shared_copies;   /* (shared node, block) pairs */
    int64_t n_sched_rounds;    /* 32-lane rounds of the node schedules */
    int64_t n_colors;          /* colours (coloured variant), else 0 */
    int64_t bandwidth_input;   /* max |i - j| over element node pairs, caller order */
    int64_t bandwidth_internal;/* the same in the library's internal order */
    int64_t max_block_elems;
    int64_t device_bytes;      /* device memory held by the mesh (0 until the
                                  first call that needs the GPU) */
    int32_t precision, variant, threads, reorder;   /* threads: CTA size of the block
                                                      kernel once on the device */
    int32_t ctas_per_sm;       /* block-kernel CTAs resident per SM (0 before the
                                  first call that needs the GPU) */
    int32_t smem_per_cta;      /* dynamic shared memory of one block-kernel CTA, bytes */
    int32_t n_instances;       /* parts of a batch (fem_batch_create), else 0 */
    int32_t n_interface_faces; /* faces given to fem_set_interface (both sides) */
} fem_info;

/* Create a mesh (Section 3: unstructured four-node tetrahedra).
 *   xyz     [n_nodes][3] coordinates, m.
 *   tets    [n_tets][4] node ids; either orientation is accepted (inverted
 *           tets are re-oriented silently).
 *   mat_id  [n_tets] material index into the table of fem_set_materials.
 *   prec    arithmetic of the step: FEM_FP64, or FEM_FP32 (bulk arithmetic
 *           in FP32; energy bookkeeping always FP64).
 *   reorder 0 keep the caller's node order, 1 reverse Cuthill-McKee
 *           (Section 5.2).
 * Errors: FEM_EINVAL for n_nodes <= 0, n_tets <= 0, NULL arrays, an id out
 * of range, a repeated node in a tet, a negative mat_id, or a degenerate
 * tet (|V| < 1e-12 l^3, l the tet's mean edge length); FEM_ENOMEM.
 * No device memory is touched by this call. */
fem_status fem_mesh_create(const double *xyz, int64_t n_nodes, const int32_t *tets,
                           int64_t n_tets, const int32_t *mat_id, fem_precision prec,
                           int reorder, fem_mesh **out);

/* As fem_mesh_create, with options (opts may be NULL for defaults). */
fem_status fem_mesh_create_ex(const double *xyz, int64_t n_nodes, const int32_t *tets,
                              int64_t n_tets, const int32_t *mat_id, fem_precision prec,
                              int reorder, const fem_options *opts, fem_mesh **out);

/* Material table [n_mat].  Builds the stored element conductances
 * K^e = k V grad N_i . grad N_j (only K^e is stored, Eq. 18 and the text
 * after it) and the row-sum lumped nodal capacities C_i = sum rho c V / 4,
 * latent capacities Lc_i = sum rho L V / 4 (Section 3).
 * Errors: FEM_EINVAL for n_mat <= 0, rho/c/k <= 0 or non-finite, latent < 0,
 * T_liquidus < T_solidus with latent > 0, a mat_id >= n_mat, or a node
 * touched by two phase-change materials with different (T_solidus,
 * T_liquidus). */
fem_status fem_set_materials(fem_mesh *m, const fem_material *mats, int32_t n_mat);

/* Flux/convective boundary Gamma_q, Eq. 4: -k dT/dn = q + h (T - T_inf) on
 * each face.  faces [n_faces][3] node ids; h, T_inf [n_faces]; q [n_faces]
 * or NULL for zero flux.  Each face must be a face of exactly one tet (a
 * boundary face).  Replaces any previous boundary; n_faces == 0 makes every
 * wall adiabatic.  Faces use the consistent Galerkin face matrix
 * h A / 12 (1 + delta_ij) and load A/3 (h T_inf - q), evaluated at step n.
 * Errors: FEM_EINVAL for an id out of range, a face that is not the face of
 * exactly one tet, h < 0, or a non-finite value. */
fem_status fem_set_boundary(fem_mesh *m, const int32_t *faces, int64_t n_faces,
                            const double *h, const double *T_inf, const double *q);

/* Temperature-dependent conductivity of material mat (Eq. 9 allows K(T)):
 * a table of n (<= 16) points, T [n] ascending (K) and k [n] > 0 (W/mK),
 * linear between points and constant beyond the ends; n == 0 restores the
 * material's constant k.  Each step evaluates k at every element's mean
 * nodal temperature of step n (explicit), K^e(T) = k(T_mean) K^e(k = 1).
 * The stable step (fem_stable_dt) uses each table's largest k.  Call after
 * fem_set_materials (which clears the tables); at most 255 materials.
 * Errors: FEM_EINVAL (material out of range, bad table), FEM_ESTATE. */
fem_status fem_set_conductivity(fem_mesh *m, int32_t mat, int32_t n, const double *T,
                                const double *k);

/* Cast-mold interface (Eq. 8): two regions meshed separately meet on a
 * surface without matching nodes.  faces_a [n_a][3] are the faces of one
 * side (e.g. the casting's), faces_b [n_b][3] the other side's, each a face
 * of exactly one tet; h_a / h_b their interface heat-transfer coefficients
 * (W/m^2K, >= 0).  Every face exchanges heat like a Robin face with
 * coefficient h_i whose ambient temperature is the mean temperature of its
 * sister at step n: the face of the other side whose centroid is nearest
 * (ties to the lower index), found once here (Section 3).  The heat shows
 * in the energy account's boundary term.  n_a == n_b == 0 removes the
 * interface.  Errors: FEM_EINVAL (ids out of range, a face that is not a
 * face of exactly one tet, one side empty, h negative or not finite). */
fem_status fem_set_interface(fem_mesh *m, const int32_t *faces_a, int64_t n_a, const double *h_a,
                             const int32_t *faces_b, int64_t n_b, const double *h_b);

/* Dirichlet boundary Gamma_T, Eq. 3: nodes [n] held at temperatures T [n]
 * (their enthalpy is never updated).  Replaces any previous set; n == 0
 * clears it.  Errors: FEM_EINVAL for an id out of range or a non-finite T. */
fem_status fem_set_dirichlet(fem_mesh *m, const int32_t *nodes, int64_t n, const double *T);

/* Initial condition, Eq. 2: T0 [n_nodes].  Sets the nodal enthalpy
 * E_i = C_i T0_i + Lc_i f_l(T0_i) (the apparent-capacity formulation keeps
 * T0 itself), resets the step count, time and the energy account (U0 = sum
 * E_i).  Requires fem_set_materials (FEM_ESTATE).
 * Errors: FEM_EINVAL for a non-finite T0. */
fem_status fem_set_temperature(fem_mesh *m, const double *T0);

/* Stable explicit step (reading of Eq. 13): 2 / max_i sum_j |(K + H)_ij| / C_i
 * over non-Dirichlet nodes, K the assembled conductance (with a k(T) table:
 * at the table's largest k), H the assembled Robin and interface face
 * matrices including an interface face's coupling to its sister's nodes,
 * C the sensible lumped capacity.  Host computation.  Requires
 * fem_set_materials (FEM_ESTATE). */
fem_status fem_stable_dt(fem_mesh *m, double *dt_out);

/* Advance n_steps explicit steps of size dt (Eq. 14 in enthalpy form):
 * T_i = T(E_i); R = F - K T; E_i += dt R_i (apparent-capacity formulation:
 * T_i += dt R_i / C_app,i).  Asynchronous on the mesh's stream.  On a batch
 * every instance takes the same steps.  n_steps == 0 is a no-op.  Errors: FEM_EINVAL for n_steps < 0 or
 * dt <= 0 / non-finite; FEM_ESTATE before fem_set_materials and
 * fem_set_temperature (or fem_set_state); FEM_ECUDA. */
fem_status fem_step(fem_mesh *m, int64_t n_steps, double dt);

/* As fem_step, timing every kernel of the step with CUDA events on the
 * mesh's stream (one synchronisation per step, so use it for measurement
 * only).  ms_out [capacity] receives the summed device milliseconds of each
 * kernel over the n_steps steps, *n_used the number of kernels per step:
 * block variant {0: block step (passes 1-3), 1: shared-node update}; atomic
 * and coloured variants {0: temperatures, 1: element pass (all colours),
 * 2: node update}; with an interface (fem_set_interface) its kernel comes
 * first and the others move up by one.  Errors as fem_step; FEM_EINVAL if
 * capacity is too small. */
fem_status fem_step_profile(fem_mesh *m, int64_t n_steps, double dt, double *ms_out,
                            int32_t capacity, int32_t *n_used);

/* Partition autotuning (block variant, single meshes and batches).  For
 * each of the n candidates (block_elems[i] tets per element block, 64 ..
 * 12288; threads[i] threads per CTA, 0 = the default for that size, else
 * 128, 256, 512 or 1024; threads may be NULL = all 0) it rebuilds the
 * element-block partition, runs 2 warm-up steps and then `steps` timed
 * steps of size dt on the mesh's stream (CUDA events), and writes the
 * mean device time per step in ms to ms_out[i] (may be NULL; +inf for a
 * candidate whose blocks do not fit in shared memory).  The fastest
 * candidate's partition is kept and its index written to *best_out.
 * The state, time, step count and energy accounts after the call are
 * those before it (the timed steps are undone).  Synchronises.  n in
 * 1..64, steps >= 1, dt as for fem_step.  FEM_ESTATE for a flat variant
 * or without an initial state; FEM_EINVAL for an out-of-range candidate
 * or when no candidate fits; FEM_ECUDA / FEM_ETIMEOUT as for fem_step. */
fem_status fem_autotune(fem_mesh *m, const int32_t *block_elems, const int32_t *threads,
                        int32_t n, int32_t steps, double dt, int32_t *best_out,
                        double *ms_out);

/* Nodal temperatures T(E) [n_nodes] in the caller's order.  Synchronises.
 * FEM_EUNSTABLE if any value is non-finite (checked on the device; the
 * output is still written); FEM_EINVAL / FEM_ETIMEOUT for an error an
 * earlier asynchronous call left on the device. */
fem_status fem_get_temperature(fem_mesh *m, double *T_out);

/* Specific nodal enthalpy E_i / m_i (J/kg) [n_nodes], caller's order. */
fem_status fem_get_enthalpy(fem_mesh *m, double *h_out);

/* FP64 energy account (device reduction): out[0] = U = sum_i E_i (J),
 * out[1] = U0 at the initial condition, out[2] = cumulative heat that
 * entered through the Robin and interface faces, out[3] = latent heat not
 * yet released sum_i Lc_i f_l(T_i).  Without Dirichlet nodes U - U0 -
 * out[2] is zero up to rounding in the enthalpy formulation (only
 * approximately in the apparent-capacity one).  Synchronises.
 * FEM_EUNSTABLE if U is non-finite, or if the balance residual
 * |U - U0 - out[2]| exceeds 2 u (n + 16) S, the most that rounding can
 * give: u the unit roundoff of the mesh's precision (2^-24 FP32, 2^-53
 * FP64), n the steps since fem_set_temperature, S the larger of |U0| and
 * |U| with |U| capped at sum_i C_i T_hi + Lc_i (T_hi the highest initial
 * or effective ambient temperature T_inf - q/h of the data).  A run past
 * the stability limit crosses that bound while every value is still
 * finite.  The check is made in the enthalpy formulation without Dirichlet
 * nodes, from fem_set_temperature (or fem_batch_create) until a state is
 * uploaded with fem_set_state*; out[] is written either way. */
fem_status fem_get_energy(fem_mesh *m, double out[4]);

/* Use the given cudaStream_t (e.g. torch.cuda.current_stream().cuda_stream)
 * for all later work of this mesh; NULL selects the legacy default stream. */
fem_status fem_set_stream(fem_mesh *m, void *cuda_stream);

/* Checkpoint: nodal enthalpy content E_i (J) [n_nodes] in the caller's
 * order, with the step count and simulated time.  Synchronises. */
fem_status fem_get_state(fem_mesh *m, double *E_out, int64_t *step, double *t);

/* Restore a checkpoint written by fem_get_state (E [n_nodes], J).
 * Asynchronous once the mesh is on the device: E is staged through a device
 * buffer on the mesh's stream; the call returns after the host-to-device
 * copy has been enqueued, so the caller must keep E unchanged until the
 * stream reaches it (any fem_get_* call guarantees that).  The energy
 * account (U0, boundary heat) is not changed.  Errors: FEM_EINVAL for
 * non-finite E -- detected on the device and returned by the next fem_get_*
 * call (before the mesh is on the device: by this call). */
fem_status fem_set_state(fem_mesh *m, const double *E, int64_t step, double t);

/* Pipelined host I/O.  A host loop of "upload a state, step, read the
 * temperatures back" overlaps the copies of neighbouring iterations with
 * the steps when it uses these three calls.  Each direction has two device
 * staging buffers and its own copy stream.  Events order every buffer's
 * reuse after its last reader, and the state update and the read-back
 * kernels run on the mesh's stream in call order.
 *
 * fem_set_state_async: as fem_set_state (E [n_nodes] in J, caller order;
 * step count and time), once the mesh has an initial state.  It returns
 * before the copy.  E must stay unchanged until fem_sync (or another
 * synchronising call) returns.  E should be page-locked (cudaHostAlloc,
 * cudaHostRegister, torch pin_memory) for the copy to overlap.
 *
 * fem_get_temperature_async: enqueues T(E) of the state after every
 * earlier call on this mesh, and its copy into T_out [n_nodes] (caller
 * order).  It returns before the copy.  T_out is valid after fem_sync, and
 * page-locked memory overlaps.
 *
 * fem_sync: waits for all asynchronous work of the mesh (both copy
 * streams and the mesh's stream) and reports what the device flagged:
 * FEM_EINVAL for a non-finite uploaded state, FEM_EUNSTABLE for a
 * non-finite temperature, FEM_ETIMEOUT for a bounded wait that gave up.
 *
 * Errors of the first two calls: FEM_EINVAL for NULL arguments, FEM_ESTATE
 * without materials or an initial state, FEM_ENOMEM / FEM_ECUDA for the
 * staging buffers (4 x n_nodes doubles on the device, allocated by the
 * first call). */
fem_status fem_set_state_async(fem_mesh *m, const double *E, int64_t step, double t);
fem_status fem_get_temperature_async(fem_mesh *m, double *T_out);
fem_status fem_sync(fem_mesh *m);

/* The same two calls with FP32 host arrays (E [n_nodes] in J, T_out
 * [n_nodes] in K): half the bytes over the host link.  An FP32 mesh holds
 * E and computes T in FP32, so they lose nothing there.  An FP64 mesh
 * converts. */
fem_status fem_set_state_async_f32(fem_mesh *m, const float *E, int64_t step, double t);
fem_status fem_get_temperature_async_f32(fem_mesh *m, float *T_out);

/* Plan statistics (host computation; builds the plan if needed). */
fem_status fem_mesh_info(fem_mesh *m, fem_info *out);

/* Reverse Cuthill-McKee order of a tet mesh's node graph (Section 5.2),
 * host only.  perm_out [n_nodes]: perm_out[old] = new.  bw_before /
 * bw_after (may be NULL): max |i - j| over element node pairs before and
 * after.  Errors: FEM_EINVAL for bad sizes or ids. */
fem_status fem_rcm_order(int64_t n_nodes, const int32_t *tets, int64_t n_tets,
                         int32_t *perm_out, int64_t *bw_before, int64_t *bw_after);

/* Host copies of the plan arrays, for inspection and tests.  which:
 *   0 node_new   int32 [n_nodes]      caller node -> internal node
 *   1 blocks     int32 [n_blocks][16] per block: e0, ne, f0, nf, n0, nint,
 *                                     c0, nsh, g0, ngrp, ne_pad, nf_pad, nep,
 *                                     r0, nrounds, s0
 *   2 elem_order int32 [E_pad]        padded element position -> caller
 *                                     element (-1 for padding)
 *   3 face_order int32 [F_pad]        padded face position -> caller face
 *   4 copy_node  int32 [n_copies]     shared copy -> internal node
 *   5 sh_ptr     int32 [n_shared+1]   shared node -> range in sh_copy
 *   6 sh_copy    int32 [n_copies]     copy indices of each shared node
 *   7 grp        int32 [..]           32-lane group -> first schedule round
 *   8 sched      uint16 [rounds*32]   slot written/read by each lane/round,
 *                                     (round r, lane) at (r/2)*64 + 2*lane + r%2;
 *                                     padding names slot 4*ne_pad + 3*nf_pad
 *   9 elem_nodes int32 [E_pad][4]     corner nodes (internal ids) per position
 *  10 face_nodes int32 [F_pad][3]     corner nodes (internal ids) per position
 *  11 copy_pos   int32 [n_copies]     position of each copy's partial sum in
 *                                     the node-ordered partial array
 *  12 block_inst int32 [n_blocks]     instance of each block (0 unless a batch)
 *  13 inst_block_start int32 [n_inst+1] first block of each instance, in plan
 *                                     order
 *  14 inst_order int32 [n_inst]       plan position -> instance
 *  15 if_sister  int32 [n_if]         sister of every interface face (index
 *                                     into side A's faces followed by side
 *                                     B's); both variants
 * *data points into the mesh (valid until the next fem_set_* or destroy);
 * *count is the number of scalar entries.  Builds the plan if needed. */
fem_status fem_plan_array(fem_mesh *m, int32_t which, const void **data, int64_t *count);

/* Energy sums of a nodal state that lives in the CALLER's device memory,
 * computed without allocating any memory.  The paper has no counterpart:
 * this serves callers that cannot call cudaMalloc -- code running while a
 * CUDA graph is being captured (an allocation there is not allowed in the
 * global capture mode), real-time loops with a no-allocation rule, or a
 * process whose device memory is owned by another allocator (for example a
 * framework's caching allocator holding the whole GPU).
 *
 *   prec    FEM_FP64 (E, C, Lc, ranges are double) or FEM_FP32 (float).
 *   E, C, Lc, phase   DEVICE arrays [n_nodes]: enthalpy content (J),
 *           sensible capacity (J/K), latent capacity (J), and a phase byte
 *           whose low 7 bits index the (Ts, Tl) pair of the node's
 *           phase-change range (ignored where Lc == 0; the high bit is
 *           ignored).  The call takes no count of pairs: wherever Lc > 0,
 *           (phase & 0x7F) must be below the number of pairs in ranges, or
 *           the kernel reads past the caller's array.
 *   ranges  DEVICE array [n_ranges][2] of (Ts, Tl).
 *   out     DEVICE array of 2 doubles: out[0] = sum_i E_i,
 *           out[1] = sum_i (E_i - C_i T(E_i)), the latent heat still held,
 *           both summed in FP64 in a fixed order (bit-reproducible).
 *   cuda_stream  stream to run on (NULL: the legacy default stream);
 *           the call is asynchronous.
 * Scratch: a static 256 KiB device array inside the library (held by every
 * GPU that loads the library until the process exits) instead of cudaMalloc.
 * All calls share it, so calls whose kernels overlap on the GPU (for
 * example on two streams at once) race and give wrong sums; serialise them.
 * Each call overwrites every scratch entry it reads, so no clearing is
 * needed.  Every call looks up the scratch's device address
 * (cudaGetSymbolAddress, no allocation) with the caller's device current,
 * so a context reset between calls is harmless.  The first call on a device
 * may load the library's device code there: make it before any stream
 * capture.
 * Errors: FEM_EINVAL for a NULL pointer, an unknown precision, or n_nodes
 * outside [1, 134217728] (the scratch holds one partial per 8192 nodes);
 * FEM_ECUDA if no device is current or the launch fails. */
fem_status fem_energy_sums_noalloc(fem_precision prec, const void *E, const void *C,
                                   const void *Lc, const uint8_t *phase, const void *ranges,
                                   int64_t n_nodes, double *out, void *cuda_stream);

/* ---- Batches: many independent meshes advanced together ------------------
 * The paper solves one casting at a time; a batch runs many castings of
 * uneven size (each with its own stable time step) on one GPU at once.  A
 * batch is an ordinary fem_mesh: every call above works on it (node, tet
 * and face ids are the concatenation of the parts': part k's node i is
 * batch node inst_node[k] + i, in part order), with these differences:
 * fem_set_materials, fem_set_boundary and fem_set_dirichlet are refused
 * (FEM_ESTATE: the parts supply them); fem_step advances every instance by
 * the same n steps of dt; fem_advance steps each instance with its own dt.
 * Element blocks never mix instances.
 */

/* Build a batch from parts (block variant, one precision; every part has
 * materials, optional boundary / Dirichlet data and an initial temperature,
 * and has not been stepped).  The parts' data are copied: the parts stay the
 * caller's and may be destroyed afterwards.  Every instance's time step
 * starts at 0.9 x its stable step (fem_instance_stable_dt).
 * Errors: FEM_EINVAL (NULL, mixed precision or variant, a part that is a
 * batch, too many distinct phase-change ranges, > 2^31 ids), FEM_ESTATE (a
 * part without materials or initial temperature, or already stepped). */
fem_status fem_batch_create(fem_mesh *const *parts, int32_t n_parts, fem_mesh **out);

/* Per-instance stable steps [n_parts] (the fem_stable_dt of each part). */
fem_status fem_instance_stable_dt(fem_mesh *m, double *dt_out);

/* Per-instance largest time steps [n_parts], s (positive, finite). */
fem_status fem_set_instance_dt(fem_mesh *m, const double *dt);

/* Advance every instance from its own current time to t_end: instance i
 * takes n_i = ceil((t_end - t_i) / dt_i) equal steps of (t_end - t_i) / n_i
 * (none if t_i >= t_end).  Each step launches the block and shared-node
 * kernels for the instances still stepping; the whole advance is captured
 * into one CUDA graph, reused while the per-instance step counts repeat.
 * Asynchronous on the mesh's stream (when that is the legacy default
 * stream, the graph runs on a library stream and the call waits for it).
 * Errors: FEM_ESTATE (not a batch, no initial state), FEM_EINVAL (t_end not
 * finite), FEM_ECUDA. */
fem_status fem_advance(fem_mesh *m, double t_end);

/* Per-instance times [n_parts] (s) and step counts [n_parts]; either
 * pointer may be NULL. */
fem_status fem_get_instance_times(fem_mesh *m, double *t_out, int64_t *steps_out);

/* Energy account of one instance, as fem_get_energy: out[0] = U (sum of
 * its nodes' E, J), out[1] = U0 (at its initial temperature), out[2] =
 * heat that entered through its Robin faces, out[3] = latent heat it still
 * holds; FP64.  Synchronises (reads the state back to the host). */
fem_status fem_get_instance_energy(fem_mesh *m, int32_t inst, double out[4]);

/* Device memory from the caller's allocator instead of cudaMalloc (for
 * example a framework's caching allocator, so that one pool serves both).
 * alloc(bytes, ctx) returns device memory on the current device, 256-byte
 * aligned (FEM_EINVAL otherwise), or NULL (FEM_ENOMEM); free_fn(ptr, ctx)
 * returns it; both are called on the thread that calls the library, while
 * the mesh's device memory is (re)built and when it is released.  Set
 * before the first call that needs the GPU (FEM_ESTATE afterwards); NULL
 * for both restores cudaMalloc. */
typedef void *(*fem_alloc_fn)(size_t bytes, void *ctx);
typedef void (*fem_free_fn)(void *ptr, void *ctx);
fem_status fem_set_allocator(fem_mesh *m, fem_alloc_fn alloc, fem_free_fn free_fn, void *ctx);

/* ---- Learned surrogate: 16 explicit steps per network evaluation -------
 * The explicit step is bounded by the stability limit of Eq. 13; a small
 * message-passing network on the node graph of the mesh advances the
 * nodal enthalpy by 16 steps of the mesh's dt in one evaluation.  The
 * paper has no surrogate: this is the library's addition, trained on
 * trajectories of the library's own explicit solver, which stays the
 * fallback and the judge of the surrogate's error.
 *
 * Graph: nodes are the mesh nodes; an edge joins two nodes of one tet, with
 * weight W_ij = -sum_e K^e_ab over the tets that hold it (Eq. 9), so that
 * sum_j W_ij (T_j - T_i) is the conduction part of the explicit residual.
 * s_i = dt_i / C_i; hA_i = sum h A / 3 and g_i = sum A (h T_inf - q) / 3 over
 * the node's Robin faces (Eq. 4 lumped to its row sums).
 * Features x_i (16; T = T(E) of Eqs. 5 and 11, f = (E - C T) / Lc the liquid
 * fraction, 0 without latent heat):
 *   (T - 600)/300, f, Lc/(300 C), 16 s hA, 16 s (g - hA T)/300,
 *   16 s sum_j W_ij (T_j - T_i)/300, 16 s sum_j W_ij (f_j - f_i), 1,
 *   (T - Ts)/300 and (T - Tl)/300 (phase-change nodes, else 0),
 *   16 s sum_j W_ij, 0 x 5.
 * Network (BF16 operands on the tensor cores, FP32 accumulation):
 *   h0 = relu(W_in x + b_in)                                16 -> 64
 *   l = 1..3: phi = relu(P_l h + p_l)                       64 -> 32
 *             m_i = s_i sum_j W_ij (phi_j - phi_i)          (FP32 sums)
 *             h  += relu(U_l [h; m] + u_l)                  96 -> 64
 *   z = relu(D1 h + d1), y = d2 . z + d2b,  E'_i = E_i + 10 K * C_i y_i.
 * Parameters: one FP32 vector of FEM_SG_N_PARAMS values, in this order:
 *   W_in [64][16], b_in [64], then for l = 1..3: P_l [32][64], p_l [32],
 *   U_l [64][96], u_l [64]; then D1 [64][64], d1 [64], d2 [64], d2b [1]
 *   (matrices row-major, out x in).
 * Training: loss = mean_i (y_i - y*_i)^2, y*_i = (E*_i - E_i) / (10 K C_i)
 * with E* the state 16 explicit steps later; Adam (b1 0.9, b2 0.999,
 * eps 1e-8) on the FP32 vector.
 * Scope: FP32 block-variant meshes in the enthalpy formulation with
 * constant conductivity, Robin faces, no Dirichlet nodes and no interface
 * faces (FEM_EINVAL otherwise).  Device arrays named E_* below are FP32
 * [n_nodes] in the surrogate's own node order (fem_surrogate_order); work
 * runs on the mesh's stream, asynchronously unless stated.  The surrogate
 * belongs to its mesh: destroy it first. */
#define FEM_SG_N_PARAMS 30177
typedef struct fem_surrogate fem_surrogate;

/* Build the graph of a mesh that has materials, boundary and a state (its
 * device data are uploaded if needed).  dt: the explicit step of a plain
 * mesh (> 0); a batch uses each instance's current step (fem_set_instance_dt)
 * and ignores dt.  Errors: FEM_EINVAL (scope above, bad dt), FEM_ESTATE,
 * FEM_ENOMEM, FEM_ECUDA. */
fem_status fem_surrogate_create(fem_mesh *m, double dt, fem_surrogate **out);

/* Sizes: nodes, directed edges (non-zeros of the graph), parameters. */
fem_status fem_surrogate_info(fem_surrogate *s, int64_t *n_nodes, int64_t *n_edges,
                              int64_t *n_params);

/* caller_of [n_nodes]: the caller's node id at each surrogate position. */
fem_status fem_surrogate_order(fem_surrogate *s, int32_t *caller_of);

/* Parameters from / to a host array of n == FEM_SG_N_PARAMS floats.
 * Setting them resets the Adam moments and step count.  Synchronises. */
fem_status fem_surrogate_set_params(fem_surrogate *s, const float *theta, int64_t n);
fem_status fem_surrogate_get_params(fem_surrogate *s, float *theta, int64_t n);

/* The mesh's current state into E_dev (device), or E_dev into the mesh
 * (the step count and time are kept; the energy account stops balancing). */
fem_status fem_surrogate_read_state(fem_surrogate *s, float *E_dev);
fem_status fem_surrogate_write_state(fem_surrogate *s, const float *E_dev);

/* E_out = the network's state 16 steps after E_in (device arrays). */
fem_status fem_surrogate_predict(fem_surrogate *s, const float *E_in, float *E_out);

/* One training step on the pair (E_in, E_star) (device arrays): forward,
 * loss, backward, then an Adam step of size lr (lr == 0: gradient only,
 * parameters unchanged).  loss_out (host, may be NULL) receives the loss
 * of the parameters before the step; a non-NULL loss_out synchronises.
 * FEM_ETIMEOUT if a bounded device wait gave up. */
fem_status fem_surrogate_train_step(fem_surrogate *s, const float *E_in, const float *E_star,
                                    float lr, double *loss_out);

/* Training over several pairs per step: fem_surrogate_accumulate runs the
 * forward and backward pass of one pair (as fem_surrogate_train_step) and
 * adds its gradient to an accumulator (loss_out as there);
 * fem_surrogate_apply takes one Adam step of size lr > 0 with the mean of
 * the accumulated gradients and clears them (FEM_ESTATE if none).
 * fem_surrogate_train_step refuses to run while gradients are pending. */
fem_status fem_surrogate_accumulate(fem_surrogate *s, const float *E_in, const float *E_star,
                                    double *loss_out);
fem_status fem_surrogate_apply(fem_surrogate *s, float lr);

/* Advance the mesh by 16 * n_macro explicit steps through the network:
 * its state is read, stepped n_macro times and written back; the step
 * count and time (each batch instance's with its own dt) advance, and the
 * energy account no longer balances (the boundary heat of those steps is
 * not accumulated). */
fem_status fem_surrogate_advance(fem_surrogate *s, int64_t n_macro);

/* Surrogate stepping with the explicit solver as judge and fallback (plain
 * meshes only).  Advances 16 * n_macro steps.  Macro step 0 is judged (if
 * judge_every > 0; 0: never judge, the surrogate takes every step): the
 * explicit solver takes the 16 steps and the surrogate's prediction from
 * the same state is compared with its result, which is kept: d = max_i
 * |E_sg,i - E_i| / C_i, a bound on the temperature difference (dT/dE <=
 * 1/C).  If d <= tol_K (K) the surrogate takes the next judge_every - 1
 * macro steps and the one after them is judged.  If d > tol_K the solver
 * takes the next span - 1 macro steps and the one after them is judged,
 * with span = judge_every * 2^min(f - 1, 6) after the f-th consecutive
 * failure (a surrogate that keeps failing is tried less and less often).
 * stats [3] (may be NULL): macro steps by the surrogate, by the solver
 * (judged ones included), judged steps that failed; max_err (may be
 * NULL): the largest d seen.  Synchronises at every judged step.  Errors
 * as fem_step and fem_surrogate_advance; FEM_EINVAL for a batch or tol_K
 * <= 0. */
fem_status fem_surrogate_solve(fem_surrogate *s, int64_t n_macro, int32_t judge_every,
                               double tol_K, int64_t *stats, double *max_err);

/* As n_macro forward passes from the mesh's state (left unchanged), with
 * CUDA events around the kernels on the mesh's stream: ms_out [5] gets the
 * summed device milliseconds of {T(E), liquid fraction and features,
 * encoder, the three message sums, the dense parts of layers 1 and 2,
 * layer 3 with the decoder}.  Measurement only. */
fem_status fem_surrogate_profile(fem_surrogate *s, int64_t n_macro, double *ms_out);

/* Test hook: a host copy of an internal buffer after the last forward or
 * training step (surrogate order).  which: 0 x (bf16 [n][16]), 1 h_layer
 * (bf16 [n][64], layer 0..3), 2 phi (bf16 [n][32], layer 0..2), 3 m (bf16
 * [n][32]), 4 relu output r (bf16 [n][64]), 5 z (f32 [n][64]), 6 y (f32
 * [n]), 7 gradient (f32 [FEM_SG_N_PARAMS]), 8 node data (f32 [n][5]: C, Lc,
 * s, hA, g), 9 graph (int32 rowptr [n+1], int32 col [n_edges], f32 w
 * [n_edges], concatenated).  bf16 values are raw 16-bit patterns.  The
 * training-only buffers (x, m, r, z, y) hold the last training step's
 * values.  Synchronises. */
fem_status fem_surrogate_debug(fem_surrogate *s, int32_t which, int32_t layer, void *out);

/* Release the surrogate's device memory (NULL is a no-op). */
void fem_surrogate_destroy(fem_surrogate *s);

/* Message of the last error on this thread ("" if none). */
const char *fem_last_error(void);

/* Release the mesh and its device memory (NULL is a no-op). */
void fem_mesh_destroy(fem_mesh *m);

#ifdef __cplusplus
}
#endif
#endif /* FEM_H */
