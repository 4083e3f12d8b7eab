/*
 * cgks.h -- C ABI of the B300 GMG-CGKS library: one pseudo-time iteration of
 * the three-level geometric-multigrid compact gas-kinetic scheme on
 * unstructured simplex meshes (Liu, Ji, Fu, Xu, "A Geometric Multigrid-
 * Accelerated Compact Gas-Kinetic Scheme for Fast Convergence in High-Speed
 * Flows on GPUs", arXiv 2509.06347).
 *
 * Conventions
 *  - Every function returns an int status: CGKS_OK (0) or a negative code.
 *    Nothing throws across the ABI.  cgks_last_error(h) returns a message that
 *    stays valid until the next call on h.
 *  - dim = 2 (triangles) or 3 (tetrahedra); nv = dim + 2 conservative
 *    variables (rho, rho u, rho v, [rho w], rho E).
 *  - Per-cell arrays exchanged through the ABI are in the ORIGINAL cell order
 *    of the uploaded mesh, row-major: W [n][nv], slopes [n][nv][dim]
 *    (d/dx_d of variable v), DF factor [n].  Internally cells are renumbered
 *    colour by colour.
 *  - Pointers flagged "on_device" are CUDA device pointers (e.g. a torch
 *    tensor's data_ptr) borrowed for the duration of the call; otherwise host
 *    pointers.  Inputs are copied; the library owns all of its state.
 *  - All work is enqueued on the stream given to cgks_create (a borrowed
 *    handle, e.g. torch.cuda.current_stream().cuda_stream).  If that handle is
 *    0 (the legacy default stream) the library uses a private stream instead.
 *    Calls that return host data synchronise that stream.
 *  - Meshes are identified by a caller-chosen integer mesh_id; several meshes
 *    can live in one context (batched solves).
 */
#ifndef CGKS_H
#define CGKS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  CGKS_OK = 0,
  CGKS_ERR_ARG = -1,         /* invalid argument, size or id */
  CGKS_ERR_MESH = -2,        /* non-manifold / open / degenerate mesh or hierarchy */
  CGKS_ERR_CUDA = -3,        /* a CUDA call failed (message in cgks_last_error) */
  CGKS_ERR_DIVERGED = -4,    /* non-finite update or residual growth beyond the limit */
  CGKS_ERR_NONPOSITIVE = -5, /* density or pressure could not be kept positive */
  CGKS_ERR_TIMEOUT = -6,     /* a bounded device wait gave up */
  CGKS_ERR_STATE = -7        /* call out of order (e.g. no mesh or state yet) */
};

/* V-cycle precision modes */
enum {
  CGKS_PLAIN_FP64 = 0, /* everything in FP64 */
  CGKS_MIXED = 1,      /* LU-SGS sweeps and their corrections in FP32; residuals,
                          DF factor and state updates in FP64 */
  CGKS_LEARNED = 2     /* MIXED fine steps, then the network's predicted coarse
                          correction where the DF factor >= cfg.df_gate instead
                          of the coarse levels; plain V-cycle fallback (2-D) */
};

/* boundary tags */
/* boundary tags: slip (inviscid) wall; far field (free stream on inflow faces,
 * interior state on outflow faces); no-slip adiabatic wall (Navier-Stokes);
 * far field from the Riemann invariants along the normal (subsonic faces take
 * the outgoing invariant from the interior, the incoming one from the free
 * stream, tangential velocity and entropy from upstream; supersonic faces the
 * upwind state) */
enum { CGKS_TAG_WALL = 1, CGKS_TAG_FARFIELD = 2, CGKS_TAG_NOSLIP_WALL = 3, CGKS_TAG_FARFIELD_RIEMANN = 4 };

typedef struct cgks_config {
  double gamma;           /* ratio of specific heats (1.4) */
  double cfl_imp;         /* CFL of the implicit (DF-weighted) part, Sec 4.3 (10); > 0 */
  double cfl_exp;         /* CFL of the explicit part and of the flux time step (0.5); > 0 */
  double tau_c1, tau_c2;  /* numerical collision time tau = c1 dt + c2 |dp|/(pl+pr) dt (0.01, 1);
                             with mu > 0 the c1 dt term gives way to mu / p; c1 > 0 and
                             c2 >= 0, finite, or cgks_create returns CGKS_ERR_ARG */
  double weno_gamma_high; /* linear weight of the large HWENO stencil (0.95) */
  double weno_eps;        /* WENO epsilon (1e-15); > 0, it keeps the weights' denominators
                             positive on flat stencils */
  double r_safety;        /* spectral-radius factor of the LU-SGS splitting (1) */
  int n_sweep_coarse;     /* LU-SGS smoothing steps per coarse level (6) */
  int n_pre, n_post;      /* fine pre/post smoothing steps (1, 0; only these are supported) */
  int check_every;        /* V-cycles between convergence checks in cgks_vcycle (10) */
  double tol;             /* residual drop that stops cgks_vcycle (1e-10) */
  double diverge_factor;  /* residual growth over the first cycle that aborts (1e6) */
  int fine_smoother;      /* 0: one DF-relaxed multi-colour LU-SGS step driven by the
                             third-order residual; 1: explicit local-time-step update
                             W -= dt_exp R / V (Eq. smo) (0) */
  int df_relax;           /* 1: DF-weighted implicit/explicit LU-SGS (Sec 4.3); 0: fully
                             implicit LU-SGS, DF ignored (ablation); 2: the fixed-factor
                             relaxation of Sec 4.3's remark, relax_beta in place of DF (1) */
  int df_prolong;         /* 1: prolongation scaled by DF (Eq. prolongation); 0: plain
                             injection (ablation) (1) */
  double df_gate;         /* learned correction applied only where DF >= df_gate (0.9) */
  int learned_judge_every;   /* plain judge cycle every this many learned-mode cycles; 0 = never (20) */
  double learned_max_error;  /* judge relative RMS error above which the network is disabled (0.5) */
  int flux_precision;        /* fine gas-kinetic flux: 0 FP64; 1 double-word (two floats, ~48-bit
                                significand, about 3.6e-15 unit roundoff) on the FP32 pipes (0) */
  double relax_beta;         /* constant relaxation factor of df_relax 2, in [0, 1] (0.5) */
  double mu;                 /* dynamic viscosity: 0 solves the Euler equations (tau = C1 dt +
                                C2 |dp|/(pl+pr) dt); mu > 0 the Navier-Stokes equations with
                                Pr = 1 (Sec 2.1): tau = mu / p + C2 |dp|/(pl+pr) dt on the fine
                                level, p that of the interface equilibrium (0) */
  double slope_relax;        /* under-relaxation of the pseudo-time slope update: slopes <-
                                slopes + slope_relax (DF grad_new - slopes); 1 replaces them
                                (Sec 2.4, 3.3).  A steady state is a fixed point for any
                                value in (0, 1] (1) */
  double alpha_relax;        /* under-relaxation of the stored DF factor: DF <- DF +
                                alpha_relax (prod of the Gauss-point factors - DF); 1 takes
                                the product (Sec 3.3).  Same fixed points for any value in
                                (0, 1] (1) */
  int learned_scale;         /* learned correction: 0 the network's inputs and target are
                                in free-stream units; 1 its 24 residual-type inputs and its
                                target are further divided by the cell's defect scale, its
                                dt_imp times the RMS over the variables of the last residual
                                norms of its mesh (group), so the network sees the defect
                                relative to the stage of the solve and its correction scales
                                with the residual (0) */
  int coarse_cluster_max_cells; /* a coarse level of two colours and at most this many cells
                                runs each smoothing step's cell residual, colour-0 forward
                                step and both sweep phases in one thread-block cluster (16
                                blocks where the device allows, else 8), with cluster
                                barriers between the phases instead of kernel boundaries;
                                bit-identical results, but slower on the 4,096- and
                                16,384-cell levels measured; 0 never (0) */
} cgks_config;

typedef struct cgks_ctx cgks_t;

/* Fills *cfg with the defaults listed above. */
int cgks_default_config(cgks_config* cfg);

/* Creates a context.  cfg is copied; stream is borrowed (see Conventions). */
int cgks_create(cgks_t** h, const cgks_config* cfg, void* cuda_stream);
/* Frees every library-owned resource of h.  h may be NULL. */
int cgks_destroy(cgks_t* h);
/* Message of the last failing call on h (borrowed; valid until the next call). */
const char* cgks_last_error(cgks_t* h);

/*
 * Mesh upload (Sec 2.2: cells, faces, Gauss points; Sec 3.1: the per-cell
 * constrained least-squares operator; Sec 4.1: colouring).  Host pointers,
 * copied:
 *   cell_nodes [n_cells][dim+1]       topological node ids (periodic images of
 *                                     a node share one id so faces match)
 *   cell_xyz   [n_cells][dim+1][dim]  each cell's own vertex coordinates (a
 *                                     face shared across a periodic boundary
 *                                     appears shifted by the period)
 *   bface_nodes [n_bfaces][dim], bface_tag [n_bfaces] (CGKS_TAG_*)
 * Face k of a cell is the face opposite its vertex k; that is the cell's
 * stored face order used by the colouring.  Returns CGKS_ERR_MESH for a face
 * shared by more than two cells, an open face missing from the boundary list
 * or a degenerate cell.  Replaces any previous mesh with the same id.
 */
int cgks_upload_mesh(cgks_t* h, int mesh_id, int dim, int64_t n_cells, const int32_t* cell_nodes,
                     const double* cell_xyz, int64_t n_bfaces, const int32_t* bface_nodes,
                     const int32_t* bface_tag);

/*
 * Mixed-element 3-D mesh upload (Sec 2.2: hexahedra, prisms and pyramids next
 * to tetrahedra; four Gauss points on every quadrilateral face).  Host
 * pointers, copied:
 *   cell_type [n_cells]          node count: 4 tetrahedron, 5 pyramid,
 *                                6 prism, 8 hexahedron
 *   cell_node_off [n_cells + 1]  offsets into cell_nodes / cell_xyz
 *   cell_nodes [sum]             node ids (faces match by their node sets)
 *   cell_xyz [sum][3]            each cell's own node coordinates
 *   bface_node_off [n_bfaces+1], bface_nodes (3 or 4 ids each), bface_tag
 * Node order: tetrahedron any (face k opposite node k); pyramid base 0-1-2-3
 * (cyclic), apex 4; prism triangles 0-1-2 and 3-4-5 with 3 above 0, 4 above
 * 1, 5 above 2; hexahedron 0-1-2-3 and 4-5-6-7 (cyclic), 4 above 0.  The
 * stored face order (used by the colouring): pyramid base, then the sides
 * 0-1, 1-2, 2-3, 3-0; prism bottom, top, then the sides 0-1, 1-2, 2-0;
 * hexahedron bottom, top, then the sides 0-1, 1-2, 2-3, 3-0.  Each cell is
 * the union of the tetrahedra from its node mean to its faces, a
 * quadrilateral face being the four triangles around its node mean (its area
 * vector 1/2 (v2 - v0) x (v3 - v1)).  A quadrilateral face's Gauss points
 * are the 2 x 2 Gauss-Legendre points of its bilinear surface, weighted by
 * the surface's local area element; a triangular face takes the 3-point
 * rule of the tetrahedral meshes.  Needs flux_precision 0 (the double-word
 * flux and the learned correction are not available on these meshes).
 * Errors as cgks_upload_mesh.  Replaces any previous mesh with the same id;
 * then cgks_upload_hierarchy as for simplex meshes.
 */
int cgks_upload_mesh_mixed(cgks_t* h, int mesh_id, int64_t n_cells, const int32_t* cell_type,
                           const int64_t* cell_node_off, const int32_t* cell_nodes, const double* cell_xyz,
                           int64_t n_bfaces, const int64_t* bface_node_off, const int32_t* bface_nodes,
                           const int32_t* bface_tag);

/*
 * Nested hierarchy (Sec 5.1-5.2).  parent[l-1][i] (host, copied) is the
 * level-l agglomerate containing level-(l-1) cell i, both in their original
 * numbering; n_levels counts the fine level (1..8).  Coarse volumes and
 * centres are sums over children; coarse faces are unique neighbour pairs with
 * summed area vectors; boundary faces are merged per (cell, tag).  Every level
 * is coloured (a coarse cell's neighbours in ascending id order) and
 * renumbered.  Allocates all solver buffers.
 */
int cgks_upload_hierarchy(cgks_t* h, int mesh_id, int n_levels, const int32_t* const* parent);

/*
 * Agglomeration coarsening (Sec 5.1, Eqs. hash value, virtual center and
 * skewness factor; Algorithm cell-merge) for meshes that are not nested by
 * construction.  Host-only; needs no mesh slot and touches no device memory.
 * Mesh arrays as in cgks_upload_mesh (host, read only; here a boundary tag
 * only groups a cell's boundary faces, so any value is taken).  The faces of
 * a level are its neighbour pairs and its (cell, tag) boundary groups, with
 * summed area vectors and centres weighted by fine face area.  One pass visits the
 * interior faces in (lower, higher) cell-id order, keeps each face whose hash
 * h = [23 (N_l + N_r) + N_l N_r] mod N_f is new (N_f = interior faces of the
 * level), and then merges the two cells of each kept face when neither was
 * merged in this pass, the face is not on a periodic seam, and every other
 * face of the merged cell has sin(alpha) = d.n / |d| > min_skew, d pointing
 * from the volume-weighted virtual centre to the face centre, n the outward
 * unit normal.  Boundary faces are never removed.  Coarse ids follow the
 * lowest member id.  One level is `passes` passes (1..8), each on the
 * agglomerates of the previous pass.  Outputs (host, caller-owned):
 *   parents     [(n_levels-1) * n_cells]  the array of level l (1..n_levels-1)
 *               starts at (l-1)*n_cells and holds level_cells[l-1] entries:
 *               the level-l agglomerate of each level-(l-1) cell, ready for
 *               cgks_upload_hierarchy; may be NULL when n_levels == 1
 *   level_cells [n_levels]  cells of each level (level_cells[0] = n_cells)
 * n_levels 1..8; min_skew in [-1, 1).  Returns CGKS_ERR_ARG for invalid
 * arguments and CGKS_ERR_MESH for a mesh that cgks_upload_mesh rejects.
 */
int cgks_agglomerate(cgks_t* h, int dim, int64_t n_cells, const int32_t* cell_nodes, const double* cell_xyz,
                     int64_t n_bfaces, const int32_t* bface_nodes, const int32_t* bface_tag, int n_levels,
                     int passes, double min_skew, int32_t* parents, int64_t* level_cells);

/* Sizes: out[4*l + 0..3] = cells, colours, faces, boundary faces of level l
 * (out must hold 4 * n_levels values); *n_levels receives the level count. */
int cgks_mesh_info(cgks_t* h, int mesh_id, int* n_levels, int64_t* out);

/* The stored numbering of a level (host int32, both nullable): order[k] = the
 * original id of the k-th stored cell (cells grouped by colour, ascending
 * colour, original order within a colour, so that each colour is one
 * contiguous launch); parent[i] = the agglomerate on the next level of
 * original cell i, in that level's original ids (not for the coarsest level). */
int cgks_get_hierarchy(cgks_t* h, int mesh_id, int level, int32_t* order, int32_t* parent);

/* Colour (1..Nc) of every cell of a level, original order, host int32 [n]. */
int cgks_get_coloring(cgks_t* h, int mesh_id, int level, int32_t* colors);

/* Free-stream state for the far-field boundaries of Sec 6 (free stream on
 * inflow faces, interior state on outflow faces, or the characteristic state
 * of the Riemann invariants): w [nv] (host, copied) in conservative variables
 * (rho, rho u, rho v, [rho w], rho E), the unknowns of Sec 2.2.  Replaces the
 * previous free stream of the mesh; after cgks_set_groups it replaces member
 * 0's only.  CGKS_ERR_ARG for a null pointer or unknown mesh. */
int cgks_set_freestream(cgks_t* h, int mesh_id, const double* w);

/* Initial state of the compact scheme (Sec 2.2: cell averages; Sec 2.4: cell-
 * averaged slopes): W [n][nv], slopes [n][nv][dim] (NULL = zero), original
 * order, host or device (on_device), copied.  Sets the DF factor (Sec 3.3) of
 * every cell to 1 and clears the residual history and counters.  Needs
 * cgks_upload_hierarchy first (CGKS_ERR_STATE otherwise). */
int cgks_init_state(cgks_t* h, int mesh_id, const double* W, const double* grad, int on_device);

/* Checkpoint / resume of the whole pseudo-time state of the fine level: the
 * cell averages and slopes the compact scheme evolves (Sec 2.2, 2.4) and the
 * DF factor the next reconstruction and LU-SGS step read (Sec 3.3, 4.3).
 * Arrays as in cgks_init_state; any pointer may be NULL (that part is left
 * as it is).  get_state synchronises the stream when on_device == 0.
 * set_state does not clear the residual history. */
int cgks_get_state(cgks_t* h, int mesh_id, double* W, double* grad, double* alpha, int on_device);
int cgks_set_state(cgks_t* h, int mesh_id, const double* W, const double* grad, const double* alpha,
                   int on_device);

/*
 * Residual at the current state without changing it.
 * level 0: third-order residual (Sec 2.2-2.4, Sec 3): R [n][nv] = total
 *   outward time-averaged flux of each cell, grad_new [n][nv][dim] = slopes
 *   from the time-evolved Gauss-point values (before the DF scaling), alpha
 *   [n] = product of the Gauss-point DF factors.  The previous DF factor of
 *   the state scales the Green-Gauss sub-stencil.
 * level >= 1: first-order KFVS residual of W_in [n_l][nv] (required; the
 *   outputs grad_new and alpha must be NULL).
 * Any output may be NULL.
 */
int cgks_residual(cgks_t* h, int mesh_id, int level, const double* W_in, double* R_out, double* grad_new_out,
                  double* alpha_out, int on_device);

/* Reconstructed polynomials of every fine cell at the current state:
 * out [n][nv][nc], nc = 6 (2-D) / 10 (3-D), P(X) = c0 + c_d X_d + sum_{d<=e}
 * c_de X_d X_e about the cell centroid (quadratic terms xx, xy, yy or xx, xy,
 * xz, yy, yz, zz).  Also returns the local time steps dt_exp, dt_imp [n]. */
int cgks_reconstruct(cgks_t* h, int mesh_id, double* coef_out, double* dt_exp_out, double* dt_imp_out,
                     int on_device);

/*
 * One multi-colour LU-SGS step with DF relaxation (Sec 4.2-4.3, Eqs.
 * gpu-forward-relaxation and gpu-backward-relaxation) on level `level` for
 * caller data: solves D dW + 1/2 alpha sum S [dT - r dW] = rhs forward over
 * colours 1..Nc then backward, with D = alpha (V/dt_imp + 1/2 sum S r) +
 * (1 - alpha) V/dt_exp, and applies W += dW with the positivity guard.
 * W_inout [n][nv] is updated; dW_out [n][nv] may be NULL.  mode selects the
 * sweep precision (CGKS_PLAIN_FP64 / CGKS_MIXED).
 */
int cgks_lusgs(cgks_t* h, int mesh_id, int level, int mode, double* W_inout, const double* rhs,
               const double* alpha, const double* dt_exp, const double* dt_imp, double* dW_out, int on_device);

/*
 * Fine smoothing, the pre-smoother of the V-cycle (Sec 5.2) on its own:
 * n_sweeps x (third-order residual of Sec 2.2-2.4 and 3, slope update with DF,
 * one DF-relaxed multi-colour LU-SGS step driven by -R (Sec 4.2-4.3, Eqs.
 * gpu-forward-relaxation and gpu-backward-relaxation), state update) on the
 * current fine state.  Only level 0 is accepted (CGKS_ERR_ARG otherwise);
 * coarse smoothing runs inside cgks_vcycle.
 */
int cgks_smooth(cgks_t* h, int mesh_id, int level, int n_sweeps);

/*
 * V-cycles (Sec 5.2; pre-smooth 1, post-smooth 0): residual and slope update,
 * fine LU-SGS, residual, restriction, FAS forcing, n_sweep_coarse KFVS +
 * LU-SGS steps per coarse level, DF-limited injection prolongation.  Runs up
 * to n_cycles cycles on each mesh (captured once into a CUDA graph and
 * replayed), stopping a mesh once its fine RMS density residual has dropped
 * by cfg.tol relative to its first recorded cycle (checked every
 * cfg.check_every cycles).  norms_out (host, nullable) receives
 * [n_meshes][n_cycles][nv][2] fine-level (RMS, max) of R/V at the start of
 * each cycle; entries of cycles not run are set to -1.  cycles_done (host,
 * nullable) [n_meshes].
 */
int cgks_vcycle(cgks_t* h, const int* mesh_ids, int n_meshes, int n_cycles, int mode, double* norms_out,
                int* cycles_done);

/* Residual norms of the last fine residual evaluation, the quantity whose
 * drop the convergence histories of Sec 6 follow (the paper plots it; the RMS
 * of the density residual per unit volume is taken here): out (host) [nv][2]
 * = RMS and max over cells of R/V.  Level 0 only.  Synchronises the stream. */
int cgks_residual_norms(cgks_t* h, int mesh_id, int level, double* out);

/* Event counters since init_state (host uint64 [4]): reconstruction
 * positivity fallbacks, halved updates, dropped updates, non-finite updates. */
int cgks_counters(cgks_t* h, int mesh_id, uint64_t* out);

/* Point evaluations for parity checks, device pointers, local frame (normal
 * = first velocity component): Wl, Wr [n][nv]; Gl, Gr [n][dim][nv] derivatives
 * along (n, t1, t2); dt [n].  Outputs F (time-averaged flux), Wt (point value
 * at t = dt) [n][nv] and the DF point factor alpha [n].  The collision time
 * follows the context's configuration (tau_c1, tau_c2, mu). */
int cgks_gks_points(cgks_t* h, int dim, int64_t n, const double* Wl, const double* Gl, const double* Wr,
                    const double* Gr, const double* dt, double* F, double* Wt, double* alpha);
/* First-order KFVS flux of constant states, device pointers [n][nv]. */
int cgks_kfvs_points(cgks_t* h, int dim, int64_t n, const double* Wl, const double* Wr, double* F);

/* Profiling hook: enqueues one stage of the fine residual at the current
 * state on the library stream (no synchronisation): 0 = reconstruction and
 * time steps, 1 = gas-kinetic face fluxes, 2 = gather.  Stage 1 needs stage 0
 * of the same state to have run. */
int cgks_run_stage(cgks_t* h, int mesh_id, int stage);

/* Number of kernel launches in one captured V-cycle of mesh_id in `mode`
 * (captures the graph if needed). */
int cgks_launch_count(cgks_t* h, int mesh_id, int mode, int* count);

/* Enqueues n_cycles V-cycles of each mesh (the captured graph) on the stream
 * without synchronising or checking convergence; the per-cycle norms are
 * recorded on the device as in cgks_vcycle. */
int cgks_vcycle_launch(cgks_t* h, const int* mesh_ids, int n_meshes, int n_cycles, int mode);

/* Check of the double-word arithmetic used by flux_precision 1 (no paper
 * counterpart): a, b (host, [n]) are split into double-words on the GPU and
 * out (host, [n][7]) receives, converted back to FP64, a + b, a - b, a * b,
 * a / b, sqrt(a), exp(-a), erfc(b).  Requires a > 0, b != 0, values within the
 * float exponent range.  Synchronises the stream. */
int cgks_dword_selftest(cgks_t* h, int64_t n, const double* a, const double* b, double* out);

/* Check of the exponential and complementary error function of the
 * half-space moments and time integrals (no paper counterpart; Sec 2.3 uses
 * exp and erfc): for x (host, [n]) out (host, [n][5]) receives erfc(x) as the
 * flux computes it (exp(-x^2) times the piecewise-polynomial erfcx),
 * erfcx(|x|), exp(-|x|) as the flux computes it, and the CUDA library's
 * erfc(x) and exp(-|x|) for comparison.  n < 2^31.  Synchronises the stream. */
int cgks_special_selftest(cgks_t* h, int64_t n, const double* x, double* out);

/* Arithmetic-throughput probe: independent FMA chains on every SM (precision
 * 0 = FP64, 1 = FP32); *tflops receives the rate measured with CUDA events.
 * Synchronises the stream.  Used as the ALU roofline denominator. */
int cgks_fma_probe(cgks_t* h, int precision, double* tflops);

/*
 * Batched solves.  After uploading the union of several meshes (disconnected
 * components, e.g. from concatenated inputs) as one mesh, tag each fine cell
 * (original order) with its member index 0..n_groups-1 and give each member
 * its own free stream winf [n_groups][nv] (host, copied).  Every coarse cell
 * must lie inside one member.  All members then advance together in every
 * launch of the V-cycle: each colour phase covers that colour of every member.
 */
int cgks_set_groups(cgks_t* h, int mesh_id, int n_groups, const int32_t* group_of_cell, const double* winf);

/*
 * V-cycles of a grouped mesh: up to n_cycles cycles; every cfg.check_every
 * cycles each member whose RMS density residual has dropped by cfg.tol from
 * its first recorded cycle is frozen (its state no longer changes) and its
 * cycle count stored in cycles_to_tol [n_groups] (-1 if not reached).  A
 * member whose residual becomes non-finite or grows by cfg.diverge_factor is
 * frozen as well, with cycles_to_tol -2; the members share no faces, so the
 * others continue unaffected.  Stops when every member is frozen.  Returns
 * CGKS_ERR_DIVERGED (after the run) if any member diverged, else CGKS_OK.
 * norms_out (host, nullable) [n_cycles][n_groups][nv][2] as in cgks_vcycle;
 * *cycles_done (nullable).
 */
int cgks_vcycle_groups(cgks_t* h, int mesh_id, int n_cycles, int mode, double* norms_out, int* cycles_to_tol,
                       int* cycles_done);

/* Autotuner: times candidate block sizes (64, 128, 256 threads) of the
 * reconstruction, flux, sweep and coarse face/cell kernels on this mesh at its
 * current state and keeps the fastest; blocks_out (nullable) [7] receives the
 * chosen sizes (reconstruction, flux, gather, sweep, coarse face, coarse cell,
 * update).  Captured graphs are rebuilt on the next V-cycle. */
int cgks_autotune(cgks_t* h, int mesh_id, int* blocks_out);

/*
 * Coarse-level KFVS residual that allocates nothing.  (The paper has no
 * counterpart; this is a service to callers.)  Same result as
 * cgks_residual(h, mesh_id, level, W, R, NULL, NULL, 1) for level >= 1, for
 * callers that cannot let a call allocate device memory, e.g. an application
 * that has planned all GPU memory up front, or a latency-critical loop where
 * cudaMalloc / cudaFree would add an implicit device synchronisation.
 *   W_dev [n_level][nv] (device, original coarse-cell order, read),
 *   R_dev [n_level][nv] (device, original order, written): outward KFVS flux
 *   of each coarse cell.
 * Stream contract: both kernels are enqueued on the context's stream and the
 * call returns without synchronising.  W_dev must be complete, and nothing
 * else may still be writing R_dev, when that stream reaches them; a caller
 * whose buffers come from work on another stream (e.g. torch's current stream
 * when the context uses its private stream) must order the two, for instance
 * by creating the context on torch's current stream or by synchronising first.
 * The per-face fluxes go to a fixed device array of 131,072 faces x 5 FP64
 * values (5 MiB) that every GPU loading the library holds until process exit;
 * levels with more faces are rejected with CGKS_ERR_ARG.  The call runs on the
 * device that was current at cgks_create (it makes that device current for
 * its duration and then restores the caller's).  The first call on each
 * context looks up that array's device address (cudaGetSymbolAddress), so make
 * the first call on a context before any stream capture.  The address is kept
 * by the context; after a device reset the context is invalid, like all of its
 * device buffers, and a new context must be created.  All calls share the
 * array: calls that overlap on the GPU (other streams, other contexts of this
 * library) race and must be serialised by the caller.
 */
int cgks_residual_coarse_noalloc(cgks_t* h, int mesh_id, int level, const double* W_dev, double* R_dev);

/*
 * Learned coarse-grid correction (a per-cell network predicting the correction
 * the coarse levels would make).  The paper has no learned component; the
 * network, its inputs and its training are this library's design.
 * Network: 76 inputs -> 64 -> GELU -> 64 -> GELU -> 4, parameters as one flat
 * FP32 vector of 9,348 values [W1 (64x76 row-major), b1, W2 (64x64), b2,
 * W3 (4x64), b3] (FP32 master copy, BF16 compute copy, FP32 accumulation).
 */
int cgks_mlp_set_params(cgks_t* h, const float* theta /* host [9348]; resets Adam */);
int cgks_mlp_get_params(cgks_t* h, float* theta /* host [9348] */);
/* Inference on device rows: X bf16 [n][76] (uint16 bit patterns), P fp32 [n][4]. */
int cgks_mlp_forward(cgks_t* h, int64_t n, const uint16_t* X, float* P);
/* Forward implementation of every later network evaluation on h (inference,
 * learned cycles and training): 0 (default) = one fused kernel per 128 rows,
 * layers 1-2 as tcgen05.mma with FP32 accumulators in tensor memory and layer
 * 3 on the CUDA cores; 1 = the mma.sync GEMM chain.  Same arithmetic (BF16
 * operands, FP32 sums) up to the order of the sums.  A tensor-core forward
 * whose bounded wait for its MMAs gives up is reported as CGKS_ERR_TIMEOUT by
 * the next cgks_synchronize, cgks_mlp_train or learned cgks_vcycle. */
int cgks_mlp_select(cgks_t* h, int impl);
/* Mean-squared-error gradient at device rows X [n][76] (bf16), Y [n][4] (fp32):
 * grad (device fp32 [9348]); loss (host, nullable). */
int cgks_mlp_grad(cgks_t* h, int64_t n, const uint16_t* X, const float* Y, float* grad, float* loss);
/* Training set held by the library: append rows (host or device pointers),
 * query its size, clear it.  An appended row with a non-finite input or
 * target (collected from a diverging mesh) is kept but takes no part in
 * training: its inputs are zeroed and it adds neither loss nor gradient. */
int cgks_mlp_dataset_append(cgks_t* h, int64_t n, const uint16_t* X, const float* Y);
int cgks_mlp_dataset_size(cgks_t* h, int64_t* n);
int cgks_mlp_dataset_clear(cgks_t* h);
/* n_steps Adam steps (beta 0.9 / 0.999, eps 1e-8) on seeded random
 * mini-batches of `batch` rows of the training set; losses (host, nullable)
 * [n_steps] receives each step's mini-batch loss. */
int cgks_mlp_train(cgks_t* h, int n_steps, int batch, double lr, uint64_t seed, float* losses);

/* Runs n_cycles plain V-cycles of a 2-D mesh (advancing its state) and
 * appends, for every cycle and fine cell, the network input (taken after the
 * fine smoothing step) and the coarse correction the cycle then applied
 * (scaled by the free stream) to the training set. */
int cgks_mlp_collect(cgks_t* h, int mesh_id, int n_cycles, int mode);

/* The network input of every fine cell at the current state of a 2-D mesh:
 * X_out (host, [n][76] bfloat16 bit patterns, original cell order).  Per cell
 * 17 values scaled by the free stream's rho, rho c, rho c, rho c^2: W (4),
 * slopes times |Omega|^(1/2) (8), R dt_imp / |Omega| (4) and the DF factor,
 * for the cell and then its 3 face neighbours in stored face order (face k
 * opposite vertex k); across a boundary face the ghost state and slopes, zero
 * residual and the cell's own DF factor and size.  Then 8 more: the fine
 * residual summed over the cell's level-1 parent and over its level-2
 * grandparent (the restriction of Sec 5.2), each times dt_imp
 * (|Omega_I| / |Omega|)^(1/2) / |Omega_I| and scaled like W (zero on meshes
 * of fewer than 3 levels).  With learned_scale 1 the 24 residual-type values
 * are further divided by the cell's defect scale (see cgks_config).  R,
 * dt_imp and DF come from a residual evaluation at the current state (as
 * cgks_residual; the state is not changed; with learned_scale 1 the
 * evaluation also sets the norms cgks_residual_norms returns).  Needs
 * cgks_mlp_set_params. */
int cgks_mlp_features(cgks_t* h, int mesh_id, uint16_t* X_out);

/* Learned-cycle statistics of the last cgks_vcycle(..., CGKS_LEARNED, ...):
 * out[10] = learned cycles, plain cycles, judge cycles, stall fallbacks,
 * network disabled (0/1), last judge relative RMS error (-1 if none), then
 * that judge's relative RMS error per conserved variable (rho, rho u, rho v,
 * E; -1 if none), each in free-stream units.
 * Policy: every 20th cycle (0, 20, 40, ...) is a plain "judge" cycle that also measures the
 * network's error against the plain correction over gated cells (disabled
 * above 0.5); a drop below 1 % over 5 learned cycles, or growth above 1.5x
 * over one cycle, switches to 10 plain cycles. */
int cgks_learned_stats(cgks_t* h, int mesh_id, double* out);

/* Waits for all work of h on its stream. */
int cgks_synchronize(cgks_t* h);

#ifdef __cplusplus
}
#endif
#endif /* CGKS_H */
