/*
 * moc_gb300.h -- C ABI of the GB300 (sm_103a) planar flat-source Method of Characteristics
 * library: 2D unstructured triangle meshes, multigroup k-eigenvalue and fixed-source transport.
 *
 * The operations follow the paper "Verification and Performance Assessment of NuDEAL, a
 * GPU-accelerated Deterministic Transport Framework on Unstructured Meshes":
 *   - multigroup transport with isotropic scattering and fission source, Eq. (MGNTE) and its
 *     element-wise form Eq. (MGNTE_element) (Sec. 2);
 *   - each triangle is one flat source region (Sec. 2.1);
 *   - characteristic solution along a segment, Eq. (MOC_sol) (Sec. 2.1);
 *   - scalar flux by angular integration over all discrete directions (Sec. 2.1);
 *   - half-edge mesh traversal, modular rays over the domain bounding box and ray-mesh
 *     intersection precomputed once (Sec. 3.1);
 *   - ray-centric GPU sweep over all rays and angles at once for isotropic scattering (Sec. 3.1);
 *   - power iteration: the fine-mesh MOC solve of Alg. 1, with the CMFD step optional and no HFEM.
 *
 * Conventions for every entry point:
 *   - Return value: MOC_OK (0) or a negative moc_status. A message for the last failure is kept
 *     per context and returned by moc_last_error(). Nothing throws or aborts across the ABI.
 *   - Host arrays passed in are owned by the caller, read during the call and copied; arrays
 *     passed out are caller-allocated and written during the call.
 *   - The context owns all device memory it allocates and frees it in moc_destroy().
 *   - Calls on one context are not thread-safe; separate contexts are independent.
 *   - Array layouts are C order. Regions are the triangles in input order; groups are
 *     innermost. Track arrays use the library's track order (direction-major, see
 *     moc_get_tracks()).
 */
#ifndef MOC_GB300_H
#define MOC_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct moc_ctx moc_ctx;

typedef enum {
  MOC_OK = 0,
  MOC_ERR_ARG = -1,            /* invalid argument (sizes, ids, non-finite or non-positive data) */
  MOC_ERR_CUDA = -2,           /* a CUDA runtime call failed */
  MOC_ERR_OOM = -3,            /* device allocation failed */
  MOC_ERR_STATE = -4,          /* call out of order (e.g. sweep before tracks/XS), or no GPU */
  MOC_ERR_NOT_CONVERGED = -5,  /* iteration limit reached before the tolerances were met */
  MOC_ERR_NONFINITE = -6,      /* k or the flux became NaN/Inf */
  MOC_ERR_GEOMETRY = -7        /* track generation failed (non-conforming mesh, lost walk) */
} moc_status;

/* Arithmetic of the sweep.
 *   MOC_FP64       : FP64 sweep, FP64 exponential, FP64 tallies.
 *   MOC_FP32       : FP32 sweep with the library's own FP32 evaluation of 1 - exp(-tau) and
 *                    Kahan-compensated FP32 region tallies (the rounding error of every atomic
 *                    update, x - (fl(old + x) - old), accumulated in a second array and folded
 *                    in at the finalize); FP64 source normalisation, k and norms.
 *   MOC_FP32_PLAIN : as MOC_FP32 with plain FP32 atomic tallies (no compensation). */
enum { MOC_FP64 = 0, MOC_FP32 = 1, MOC_FP32_PLAIN = 2 };

/* Boundary conditions per wall of the bounding box (x-, x+, y-, y+). */
enum { MOC_BC_VACUUM = 0, MOC_BC_REFLECTIVE = 1 };
enum { MOC_RAYS_MODULAR = 0, MOC_RAYS_BACK_PROJECTION = 1 };

/* Create a context on CUDA device `device` (>= 0) with sweep arithmetic `precision`.
 * `stream` is a cudaStream_t the context launches all work on (NULL: the context creates its
 * own). device = -1 creates a host-only context: mesh, quadrature and track generation work;
 * every call that needs the GPU returns MOC_ERR_STATE.  *out is NULL on failure. */
int moc_create(moc_ctx **out, int device, int precision, void *stream);

/* Free the context and all device memory it owns. NULL is allowed. */
void moc_destroy(moc_ctx *ctx);

/* Message of the last failed call on ctx (empty if none). Valid until the next call on ctx. */
const char *moc_last_error(const moc_ctx *ctx);

/* Triangle mesh (Sec. 3.1). xy: [n_vert][2] vertex coordinates (cm); tri: [n_tri][3] vertex
 * ids, counter-clockwise; tri_material: [n_tri] material ids (checked in moc_set_xs); bbox:
 * xmin, xmax, ymin, ymax of the domain's bounding box; bc: [4] MOC_BC_* for x-, x+, y-, y+.
 * The mesh must be conforming (interior edges shared by exactly two triangles with opposite
 * orientation). Reflective walls require the mesh to fill the box along that wall.
 * Errors: MOC_ERR_ARG for bad sizes, ids, orientation or a non-conforming edge. */
int moc_set_mesh(moc_ctx *ctx, int n_vert, const double *xy, int n_tri, const int32_t *tri,
                 const int32_t *tri_material, const double *bbox, const int32_t *bc);

/* Angular quadrature. n_azim: azimuthal angles over [0, 2 pi), a multiple of 4; ray_spacing
 * (cm) > 0: the requested distance between parallel rays (the effective one is never larger);
 * sin_theta, polar_w: [n_polar] polar angles of one hemisphere and their weights (sum 1).
 * 1 <= n_polar <= 6. Errors: MOC_ERR_ARG. */
int moc_set_quadrature(moc_ctx *ctx, int n_azim, double ray_spacing, int n_polar,
                       const double *sin_theta, const double *polar_w);

/* Ray layout of the next moc_generate_tracks (Sec. 3.1 names both): MOC_RAYS_MODULAR (default),
 * cyclic rays over the bounding box with corrected angles, the only layout that can link
 * reflective walls; or MOC_RAYS_BACK_PROJECTION, rays cast from the domain boundary into the
 * mesh at the nominal angles 2 pi (a + 1/2)/n_azim (weights 1/n_azim), per direction n =
 * ceil(extent / ray_spacing) rays spread evenly (spacing extent/n, offset half a spacing) over
 * the extent of the mesh projected on the direction's normal -- no rays are spent on the empty
 * corners of a non-rectangular domain's bounding box. Back projection requires every boundary
 * to be vacuum (moc_generate_tracks returns MOC_ERR_ARG otherwise). Errors: MOC_ERR_ARG. */
int moc_set_ray_layout(moc_ctx *ctx, int layout);

/* Lay down the modular (cyclic) rays over the bounding box, intersect them with the mesh by a
 * half-edge walk, build the reflective links and the tracked region areas, and upload the
 * segment data to the device (Sec. 3.1). Readings where the paper is silent: first-quadrant
 * nominal angle 2 pi (a + 1/2)/n_azim, nx = floor(W sin/spacing) + 1, ny = floor(H cos/spacing)
 * + 1, corrected angle atan(H nx / (W ny)), ray starts at (i + 1/2) W/nx and (j + 1/2) H/ny;
 * pieces shorter than 1e-12 cm are dropped; a ray leaving a non-rectangular mesh and
 * re-entering it starts a new track with vacuum inflow.
 * Errors: MOC_ERR_STATE (no mesh/quadrature), MOC_ERR_GEOMETRY, MOC_ERR_OOM, MOC_ERR_CUDA. */
int moc_generate_tracks(moc_ctx *ctx);

/* Same as moc_generate_tracks, with the ray-mesh intersection (the half-edge walk of every ray,
 * Sec. 3.1) run on the context's GPU, one thread per ray in a counting pass and a filling pass;
 * ray laydown, boundary-entry events, links and areas stay on the host. The device walk uses the
 * host walk's code and IEEE double arithmetic without contracted multiply-adds, so tracks and
 * segments are bit-identical to moc_generate_tracks (areas, summed from the same segments, are
 * too). For fast re-tracking of large meshes. walk_ms (may be NULL) gets the device time of the
 * two passes. Errors: as moc_generate_tracks; MOC_ERR_STATE on a host-only context. */
int moc_generate_tracks_device(moc_ctx *ctx, double *walk_ms);

/* Tracks from the caller instead of moc_generate_tracks (segments computed elsewhere; the paper
 * precomputes the segment data before the sweep, Sec. 3.1). Needs moc_set_mesh (regions) and
 * moc_set_quadrature (polar set; n_azim fixes n_dir = n_azim/2 directions over [0, pi)).
 *   seg_off     [n_tracks+1] first segment of each track, seg_off[0] = 0, every track non-empty
 *   seg_region  [S] region of each segment; seg_len [S] its 2D length (finite, > 0)
 *   track_azim  [n_tracks] direction index 0..n_dir-1 of each track (swept in both senses)
 *   azim_weight [n_dir] azimuthal weight omega_j (the 2 pi set: each stands for j and j + pi)
 *   azim_spacing[n_dir] ray spacing delta_j
 *   link        [n_tracks][2] incoming end (2 t' + d') fed by the outgoing end of (t, d), or -1
 *               (vacuum); each incoming end fed at most once
 * Areas are the tracked areas sum 2 omega_j delta_j l. The directions' angles are unknown, so
 * moc_set_scattering is refused on such tracks. Arrays are copied; replaces tracks, cross
 * sections and state like moc_generate_tracks. Errors: MOC_ERR_ARG (validation), MOC_ERR_STATE,
 * MOC_ERR_OOM, MOC_ERR_CUDA. */
int moc_set_tracks(moc_ctx *ctx, int64_t n_tracks, const int64_t *seg_off, const int32_t *seg_region,
                   const double *seg_len, const int32_t *track_azim, const double *azim_weight,
                   const double *azim_spacing, const int32_t *link);

/* Number of tracks and segments after moc_generate_tracks(). */
int moc_get_track_counts(const moc_ctx *ctx, int64_t *n_tracks, int64_t *n_segments);

/* Copy out the tracks (for inspection and tests). Track order: direction index j = 0 ..
 * n_azim/2 - 1 (angles in [0, pi) ascending), for each the rays starting on the bottom edge
 * (left to right) then on the side edge (bottom to top), each ray's tracks in order along it.
 * seg_off: [T+1]; seg_region: [S]; seg_len: [S] (cm, 2D length); track_dir: [T];
 * track_xy: [T][4] start x, y, end x, y; link: [T][2] for each track end (0: forward sweep's
 * outgoing end at the track end, 1: backward sweep's at the start) the incoming end it feeds,
 * encoded 2 t' + d', or -1 for vacuum. Any output pointer may be NULL. */
int moc_get_tracks(const moc_ctx *ctx, int64_t *seg_off, int32_t *seg_region, double *seg_len,
                   int32_t *track_dir, double *track_xy, int64_t *link);

/* Quadrature after track generation: per direction j < n_azim/2 the corrected angle, the
 * effective spacing and the azimuthal weight (weights of the 2 pi set sum to 1). */
int moc_get_quadrature(const moc_ctx *ctx, double *phi, double *delta, double *omega);

/* Tracked region areas [n_tri]: A_i = sum over the 2 pi set of omega_a delta_a (length in i). */
int moc_get_region_areas(const moc_ctx *ctx, double *area);

/* Multigroup cross sections per material (Eq. MGNTE): sigma_t, nu_sigma_f, chi: [n_mat][G];
 * sigma_s: [n_mat][G_from][G_to] isotropic (P0) scattering. Requires sigma_t > 0, all data
 * finite and >= 0, sigma_t >= the total scattering out of each group (absorption >= 0), and
 * every mesh material id < n_mat. Resets the state to phi = 1, k = 1,
 * zero boundary flux, eigenvalue mode. Errors: MOC_ERR_ARG, MOC_ERR_STATE, MOC_ERR_OOM. */
int moc_set_xs(moc_ctx *ctx, int n_mat, int G, const double *sigma_t, const double *nu_sigma_f,
               const double *chi, const double *sigma_s);

/* Coarse-mesh finite difference (CMFD) acceleration of the power iteration (Alg. 1: CMFD on a
 * coarse mesh from the MOC surface currents, then the fine MOC solution updated with the
 * accelerated result). cell: [n_tri] coarse cell (0 .. n_cells-1) of every region, any partition
 * of the triangles; NULL switches the acceleration off. Partial-current form: the sweep tallies,
 * per pair of cells and direction, W * psi at every crossing between them, and per cell the net
 * current through the domain boundary (out at every track end, in at every track start, vacuum and
 * reflective walls alike); each cell's balance uses flux-volume homogenised cross sections and
 * coefficients J/phi that reproduce the MOC currents, so the converged MOC solution is unchanged.
 * After each outer the coarse eigenproblem is iterated n_outer times (Gauss-Seidel in energy;
 * per group n_inner over-relaxed Gauss-Seidel sweeps with factor omega in (0, 2), over a greedy
 * colouring of the cells in ascending id, one colour at a time), then phi and the incoming
 * boundary flux are scaled by the coarse/fine flux ratio of their cell and k becomes the coarse
 * k. Eigenvalue mode only; must be called after moc_set_xs (which switches it off). The coarse
 * solve runs in one thread block; its per-group working set is kept in shared memory when it
 * fits in what the device allows a block after 9 KB (FP32: 16 bytes per cell and 6 per interface
 * side, e.g. the 4,624 cells of a 68 x 68 grid), else in global memory. Errors: MOC_ERR_ARG,
 * MOC_ERR_STATE. */
int moc_set_cmfd(moc_ctx *ctx, const int32_t *cell, int n_cells, int n_outer, int n_inner, double omega);

/* Early stop of the CMFD coarse power iteration (a production mode; the paper fixes no coarse
 * iteration count): with tol > 0, each outer's coarse iteration ends after the first coarse
 * iteration (at most n_outer of moc_set_cmfd) whose k change is <= tol * k and whose coarse
 * fission source, normalised to unit sum, changes by <= tol relative in every cell. tol = 0, the
 * value a new context starts with, runs exactly n_outer iterations; moc_set_cmfd leaves the
 * setting as it is. The converged MOC solution does not depend on it (it is a fixed point of every
 * coarse step). Errors: MOC_ERR_ARG (tol negative or not finite). */
int moc_set_cmfd_tolerance(moc_ctx *ctx, double tol);

/* Coarse power iterations run since the last moc_set_state (or moc_set_xs), summed over outers.
 * Synchronises. Errors: MOC_ERR_ARG, MOC_ERR_STATE (host-only context), MOC_ERR_CUDA. */
int moc_get_cmfd_iterations(moc_ctx *ctx, int64_t *total);

/* Anisotropic scattering of Legendre order L (Sec. 2: the scattering kernel expanded as
 * sum_l (2l+1)/(4 pi) P_l(Om . Om') Sigma_s,l). sigma_sl: [L][n_mat][G][G] holds Sigma_s,l g -> g'
 * (from-group major, like sigma_s) for l = 1..L, 1 <= L <= 3; L = 0 or NULL restores isotropic
 * scattering (Sigma_s,0 is moc_set_xs's sigma_s). The library carries the angular moments of the
 * flux against the real harmonics with l + m even (the ones a plane problem keeps, L(L+3)/2 of
 * them): each source update builds per region and group the moments (2l+1) Sigma_s,l phi_lm;
 * the sweep uses the source of every discrete direction and tallies every moment; after the sweep
 * the moments are the discrete angular integrals of the region-average angular flux (the discrete
 * quadrature's Gram matrix, not an assumed orthogonality). set_state restarts the moments from an
 * isotropic angular flux. Up to 3 polar angles; not combined with CMFD (MOC_ERR_STATE); FP32 moment
 * tallies are plain atomic sums. Call after moc_set_xs (which switches it off). Errors:
 * MOC_ERR_ARG, MOC_ERR_STATE. */
int moc_set_scattering(moc_ctx *ctx, int L, const double *sigma_sl);

/* Fixed isotropic volumetric source S: [n_tri][G] (n/cm^3/s), switching the context to
 * fixed-source mode (fission ignored, no normalisation); NULL returns to eigenvalue mode. */
int moc_set_fixed_source(moc_ctx *ctx, const double *S);

/* Set the iterate: phi [n_tri][G] (NULL: all ones), k, psi_bnd [T][2][n_polar][G] incoming
 * angular flux per track end (NULL: zero). In eigenvalue mode the state is normalised so that
 * sum_i A_i sum_g nuSigma_f phi = 1 before the next outer. */
int moc_set_state(moc_ctx *ctx, const double *phi, double k, const double *psi_bnd);

/* Read the iterate (normalised in eigenvalue mode). Any output may be NULL. Synchronises. */
int moc_get_state(moc_ctx *ctx, double *phi, double *k, double *psi_bnd);

/* Enqueue the source update of Eq. (MGNTE_element) from the current (phi, k). Asynchronous. */
int moc_update_source(moc_ctx *ctx);

/* Enqueue one transport sweep (Eq. MOC_sol over every track, both directions, every polar
 * angle and group, tallies, boundary-flux links), the flux finalisation and the FP64 fission /
 * residual reductions, using the source from the last moc_update_source(). Asynchronous. */
int moc_sweep(moc_ctx *ctx);

/* Enqueue n outer iterations (source update + sweep each). Asynchronous; k_out and resid_out
 * (may be NULL) are read back with a synchronisation after the last outer. */
int moc_outer(moc_ctx *ctx, int n, double *k_out, double *resid_out);

/* One outer (source, sweep, finalize, k and normalisation) with the scalar flux in device arrays
 * owned by the caller (e.g. PyTorch tensors), enqueued on `stream` (a cudaStream_t; NULL = the
 * context's stream; ordered after the context's pending work and before its later work).
 *   phi_in_dev  [n_tri][G] flux the source is built from, in the context's type (float for the
 *               FP32 modes, double for FP64), taken as normalised (e.g. the phi_out of the
 *               previous call), or NULL to continue from the context's flux
 *   phi_out_dev [n_tri][G] the new flux, normalised to F = 1 in eigenvalue mode, or NULL
 * The caller keeps both alive until the stream's work completes. Asynchronous; k and the residual
 * as after moc_outer (read with moc_outer(ctx, 0, &k, &r)). Errors: MOC_ERR_STATE, MOC_ERR_CUDA. */
int moc_sweep_dev(moc_ctx *ctx, void *stream, const void *phi_in_dev, void *phi_out_dev);

/* DGMOC (Sec. 2.2 "DGMOC formulation", Eq. DGMOC_expansion to DGMOC_weak_up; Alg. 2): extrude the
 * planar tracks through nz axial planes of heights dz[nz] (cm, > 0) and solve the 3D problem with
 * a linear discontinuous-Galerkin expansion in z on every characteristic (the angular flux in
 * each plane is a + b xi, xi from -1 at the plane's bottom to +1 at its top; axial faces are
 * upwinded; the inflow of a segment is the segment average of the upwind plane's outflow trace).
 * mat3 [nz][n_regions] gives each region's material in each plane (NULL: the mesh's materials in
 * every plane). bc_bottom, bc_top: 0 vacuum, 1 reflective (a reflective bottom feeds the upward
 * march with the same sweep's bottom traces, a reflective top feeds the downward march with the
 * previous sweep's top traces). Up to 4 polar angles; each polar angle serves an upward and a
 * downward direction of weight 2 pi omega w_p delta. Call after moc_set_xs (moc_set_xs and new
 * tracks switch DGMOC off); nz = 0 switches it off. Not combined with CMFD, anisotropic
 * scattering, moc_sweep_dev or the warm start (MOC_ERR_STATE). The state restarts flat.
 * While DGMOC is on: moc_set_state / moc_get_state take phi as [nz][n_regions][2][G] (plane
 * average, then the xi coefficient of the scalar flux) and psi must be NULL (the boundary flux
 * restarts at zero); moc_set_fixed_source's [n_regions][G] source applies in every plane; every
 * other call (moc_outer, moc_power_iterate, timing, history) works as in the planar method, with
 * the fission source summed as dz A nuSigma_f phi_0 and the residual over (plane, region) elements.
 * FP32 modes tally in plain FP32 (no compensation). Errors: MOC_ERR_ARG (sizes, heights not
 * finite or below 1e-9 cm, material ids, more than 4 polar angles), MOC_ERR_STATE, MOC_ERR_OOM,
 * MOC_ERR_CUDA. */
int moc_set_axial(moc_ctx *ctx, int nz, const double *dz, const int32_t *mat3, int bc_bottom, int bc_top);

/* Axial coarse-mesh acceleration of DGMOC (the CMFD step of Alg. 1 with the planes as coarse
 * cells), eigenvalue mode: each outer's sweep also tallies the partial currents between planes and
 * each plane's net current through the domain boundary (radial track ends, bottom and top faces,
 * out minus in); the planes' flux-volume homogenised balance, with D = J / phi from those currents
 * (a fixed point at the transport solution), is iterated n_outer times (power iteration;
 * Gauss-Seidel in energy; n_inner sweeps over the even then the odd planes, over-relaxed by omega
 * in (0, 2)), and both flux moments, the next sweep's radial boundary flux and the stored top
 * traces are scaled by their plane's coarse/fine ratio; k becomes the coarse k. n_outer = 0
 * switches it off; moc_set_axial switches it off. Needs the plane-inner sweep (its shared memory
 * with the current sums must fit 100 KB per block: nz <= 22 in FP32, 11 in FP64 with 3 polar
 * angles). Errors: MOC_ERR_STATE (no moc_set_axial), MOC_ERR_ARG, MOC_ERR_OOM, MOC_ERR_CUDA. */
int moc_set_dg_cmfd(moc_ctx *ctx, int n_outer, int n_inner, double omega);

/* Iteration history: every time the host reads k and the residual after outers (each check of
 * moc_power_iterate, moc_outer with k_out or resid_out), one entry {outers so far (since the last
 * moc_set_state), k, k before the last outer, residual} is recorded; the last 4,096 are kept.
 * Copies the most recent min(max_entries, recorded) entries, oldest first, into entries
 * [n][4] and their count into *n_out. Errors: MOC_ERR_ARG. */
int moc_get_history(const moc_ctx *ctx, double *entries, int max_entries, int *n_out);

/* Average sweep time (ms) and segment-polar-group updates per second over the sweeps timed since
 * moc_enable_timing(ctx, 1) (synchronises; 0 if none). */
int moc_get_stats(moc_ctx *ctx, double *sweep_ms, double *updates_per_s);

/* Iterate until |k' - k| <= tol_k and the L-inf relative fission-source change <= tol_flux
 * (fixed-source mode: the relative flux change <= tol_flux), or max_outer outers. Convergence
 * is checked on the host every `check_every` outers (the outers in between run as one CUDA
 * graph launch). Returns MOC_ERR_ARG unless max_outer >= 1, check_every >= 1, tol_k >= 0 and
 * tol_flux >= 0 (NaN tolerances included), MOC_ERR_NOT_CONVERGED if max_outer is reached,
 * MOC_ERR_NONFINITE if k or the residual is not finite. */
int moc_power_iterate(moc_ctx *ctx, double tol_k, double tol_flux, int max_outer,
                      int check_every, double *k_out, int *n_outer_out, double *resid_out);

/* Timing of the sweep kernel, measured with CUDA events on the context's stream when enabled:
 * enable != 0 starts recording (and resets the totals); the getter returns the summed sweep
 * kernel time (ms) and the number of timed sweeps since. */
int moc_enable_timing(moc_ctx *ctx, int enable);
int moc_get_timing(moc_ctx *ctx, double *sweep_ms_total, int64_t *n_sweeps);

/* Work counters: segments S, updates per sweep 2 S P G, and the number of kernels one outer
 * launches. */
int moc_get_work(const moc_ctx *ctx, int64_t *n_segments, int64_t *updates_per_sweep,
                 int *kernels_per_outer);

/* Learned warm start, context side (the network itself is in moc_mlp.h). The paper has no
 * counterpart; the cold start (flat flux, k = 1, zero boundary flux) remains the fallback.
 *
 * moc_ws_features: per-region network inputs feat_dev [n_tri][3 G + n_geo + n_glob] =
 * (Sigma_t, nu Sigma_f, Sigma_a of the region's material) ++ geo_dev row ++ glob, built on the
 * device from the cross sections set by moc_set_xs. geo_dev: device [n_tri][n_geo] (may be NULL
 * when n_geo = 0); glob: host [n_glob]; feat_dev: device, caller-owned. Enqueued on the context's
 * stream.
 *
 * moc_ws_apply: set the iterate from a prediction pred_dev [n_tri][G + 1] (device): phi = exp of
 * the first G columns, k = area-weighted mean of the last column, incoming boundary flux of every
 * linked track end = phi of the region at that end / (4 pi) for all polar angles, vacuum ends
 * zero; then normalised as moc_set_state does. Enqueued on the context's stream; k_out (may be
 * NULL) synchronises. Errors: MOC_ERR_STATE (no tracks/XS), MOC_ERR_ARG. */
int moc_ws_features(moc_ctx *ctx, const float *geo_dev, int n_geo, const float *glob, int n_glob,
                    float *feat_dev);
int moc_ws_apply(moc_ctx *ctx, const float *pred_dev, double *k_out);

/* Evaluate the library's FP32 1 - exp(-tau) (the one the FP32 sweep uses) for n host values
 * tau[i] >= 0 into out[i], on device `device`. Host buffers; synchronous. For checking the
 * approximation error against an FP64 reference. Errors: MOC_ERR_ARG, MOC_ERR_CUDA. */
int moc_eval_one_minus_exp_f32(int device, const float *tau, float *out, int64_t n);

/* The same function in its packed form, two values per f32x2 multiply, add and fused multiply-add
 * (as the FP32 sweeps evaluate it): each component is rounded as in the scalar form, so out equals
 * moc_eval_one_minus_exp_f32's output bit for bit. Both ways the sweeps form the scale 2^-n (an
 * integer multiply-add, or a shift and subtract) are evaluated; out[i] is NaN where they differ.
 * Host buffers; synchronous. Errors: MOC_ERR_ARG, MOC_ERR_CUDA. */
int moc_eval_one_minus_exp_f32x2(int device, const float *tau, float *out, int64_t n);

/* Wait for all work enqueued on the context's stream. */
int moc_synchronize(moc_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* MOC_GB300_H */
