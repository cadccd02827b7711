/*
 * robast.h -- C ABI of the GB300 (sm_103a) non-sequential photon tracer.
 *
 * Method: Okumura, Noda, Rulten, "ROBAST: Development of a Non-Sequential
 * Ray-Tracing Simulation Library and its Applications in the Cherenkov
 * Telescope Array", ICRC 2015 (arXiv:1508.07803).
 *   Sec. 1, 2.1  non-sequential tracing: at every step the photon goes to the
 *                NEAREST intersection over all surfaces; the surface's role
 *                decides the interaction (mirror: reflect; lens: refract;
 *                focal surface: detect; obscuration: absorb); repeat until
 *                the photon terminates.
 *   Sec. 2.2     shapes: primitive shapes, the aspheric disk, the polygonal
 *                Winston cone and the Bezier-profile polygonal cone.
 *   Sec. 3       workloads: segmented dishes with masts and camera boxes,
 *                Schwarzschild-Couder aspheric two-mirror optics, hexagonal
 *                light concentrators; results are spot diagrams (PSF) and
 *                collection efficiency.
 *
 * Conventions for every call:
 *   - return 0 on success, a negative ROBAST_E* code on failure; the message
 *     of the last failure on this host thread is robast_last_error().  The
 *     library never aborts, traps or exits.  Problems of single photons
 *     (Newton non-convergence, non-finite directions, traversal stack
 *     overflow) are reported as ROBAST_ST_ERROR in that photon's status, not
 *     as a return code.
 *   - lengths in metres (any consistent unit works), wavelengths in nm,
 *     angles in radians.
 *   - "device pointer": memory the CUDA runtime can address from the GPU
 *     (cudaMalloc / torch CUDA tensors); "host pointer": ordinary memory.
 *   - vectors of n photons are SoA in ONE buffer of 3n elements: all x, then
 *     all y, then all z.  Element type is float for precision 32 and double
 *     for precision 64.
 *   - all GPU work is asynchronous on the caller's stream unless stated.
 */
#ifndef ROBAST_H
#define ROBAST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes */
#define ROBAST_OK 0
#define ROBAST_E_INVALID (-1)   /* bad descriptor or argument */
#define ROBAST_E_NULL (-2)      /* required pointer is NULL */
#define ROBAST_E_CUDA (-3)      /* CUDA runtime error */
#define ROBAST_E_OOM (-4)       /* device or host allocation failed */
#define ROBAST_E_UNSUPPORTED (-5)

/* surface shapes (Sec. 2.2) */
#define ROBAST_SHAPE_SAG 0      /* even asphere: conic + A1 r^2 .. A8 r^16 (plane, sphere, paraboloid included) */
#define ROBAST_SHAPE_CYLINDER 1 /* open finite cylinder, local z axis, 0 <= z <= length */
#define ROBAST_SHAPE_BOX 2      /* box centred at the local origin */
#define ROBAST_SHAPE_HEXCONE 3  /* hexagonal cone, quadratic-Bezier wall profile (Winston / Okumura cone) */

/* surface roles (Sec. 2.1: AMirror, ALens, AFocalSurface, AObscuration) */
#define ROBAST_ROLE_MIRROR 0
#define ROBAST_ROLE_REFRACT 1
#define ROBAST_ROLE_FOCAL 2
#define ROBAST_ROLE_OBSCURATION 3

/* apertures of a SAG surface, on the local (x, y) of the hit; edges inclusive */
#define ROBAST_AP_NONE 0    /* unbounded */
#define ROBAST_AP_CIRCLE 1  /* ap[0] = r_max */
#define ROBAST_AP_ANNULUS 2 /* ap[0] = r_min, ap[1] = r_max */
#define ROBAST_AP_SECTOR 3  /* ap[0..1] = r_min, r_max; ap[2..3] = phi0 < phi1, phi1 - phi0 <= pi */
#define ROBAST_AP_HEXAGON 4 /* ap[0] = apothem; flats face 0, 60, 120 deg of local x */
#define ROBAST_AP_RECT 5    /* ap[0] = half width in x, ap[1] = half width in y */

/* photon end states */
#define ROBAST_ST_DETECTED 1    /* front side of a focal surface */
#define ROBAST_ST_ABSORBED 2    /* lost to a mirror's reflectivity draw */
#define ROBAST_ST_OBSCURED 3    /* obscuration, or the back of a mirror / focal surface */
#define ROBAST_ST_ESCAPED 4     /* no further intersection */
#define ROBAST_ST_MAX_BOUNCES 5 /* still alive after max_bounces interactions */
#define ROBAST_ST_ERROR 6       /* Newton failure, non-finite state, stack overflow */

/* counters accumulated by robast_trace* (device uint64 array, never cleared by the library) */
#define ROBAST_CNT_BOUNCES 0  /* sum of bounce counts */
#define ROBAST_CNT_PHOTONS 7  /* photons finished; [1..6] = photons per status */
#define ROBAST_N_COUNTERS 8

/* ------------------------------------------------------------- geometry */
/*
 * One surface in its own local frame.  A world point p has local coordinates
 * R' (p - origin), where R' = Ry(tilt[1])^T Rx(tilt[0])^T R and R = rot
 * (row-major, row k = local axis k in world coordinates, orthonormal).  The
 * tilt is a rotation of the surface about its local x axis, then its local y
 * axis, through the local origin (facet alignment errors, Sec. 3).
 *
 * SAG: z = c rho / (1 + sqrt(1 - (1+k) c^2 rho)) + sum_i asph[i-1] rho^i,
 *      rho = x^2 + y^2, i = 1..8.  Front side = the side the local +z axis
 *      points to.  With any asph != 0 the intersection is found by Newton from
 *      the first on-branch root of the conic (only within 1.1x the aperture's
 *      bounding radius).
 * CYLINDER: prm[0] = radius, prm[1] = length.
 * BOX: prm[0..2] = half extents.
 * HEXCONE: prm[0..5] = (r, z) of the Bezier control points P0, P1, P2; wall j
 *      (j = 0..5) faces direction (cos j pi/3, sin j pi/3); front side = the
 *      side facing the cone axis.
 */
typedef struct robast_surface_desc {
    int32_t shape, role, aperture;
    int32_t material;                   /* MIRROR: index into materials */
    int32_t medium_front, medium_back;  /* REFRACT: media on the front / back side */
    int32_t reserved;
    double origin[3];
    double rot[9];
    double tilt[2];
    double curv, conic;
    double asph[8];
    double ap[4];
    double prm[8];
} robast_surface_desc;

#define ROBAST_MAX_TABLE 16
/* Mirror coating: reflectivity R(lambda) piecewise linear in (lam, refl),
 * clamped outside; roughness = Gaussian tilt of the normal, sigma per tangent
 * axis (rad). */
typedef struct robast_material_desc {
    int32_t n, reserved;
    double lam[ROBAST_MAX_TABLE];
    double refl[ROBAST_MAX_TABLE];
    double sigma;
} robast_material_desc;

/* Refractive medium: n_const > 0 gives a constant index, otherwise the
 * Sellmeier form n^2 = 1 + sum B_i l^2 / (l^2 - C_i), l in micrometres.
 * Bulk absorption (n_abs > 0): absorption length abs_len (m) piecewise linear
 * in abs_lam (nm), clamped; a photon that reaches a refracting face after a
 * path s through this medium (the medium on its side of that face) survives
 * with probability exp(-s / len), decided by Philox word 3 of that
 * interaction, else it is ABSORBED there. */
typedef struct robast_medium_desc {
    double n_const;
    double B[3], C[3];
    int32_t n_abs, reserved;
    double abs_lam[ROBAST_MAX_TABLE];
    double abs_len[ROBAST_MAX_TABLE];
} robast_medium_desc;

/*
 * The optical system(s).  variant_offsets (n_variants + 1 entries, NULL for a
 * single variant) splits the surface array into independent systems traced
 * side by side (batching); a photon sees only its variant's surfaces.
 * length_scale (L_sys, > 0) sets the default self-intersection epsilon.
 */
typedef struct robast_geom_desc {
    int32_t n_surfaces, n_materials, n_media, n_variants;
    const robast_surface_desc* surfaces;
    const robast_material_desc* materials;
    const robast_medium_desc* media;
    const int32_t* variant_offsets;
    double length_scale;
} robast_geom_desc;

typedef struct robast_geom robast_geom; /* opaque */

/*
 * Compile a host descriptor into device tables (per-surface frames and shape
 * records in FP32 and FP64, a BVH over surface bounding boxes per variant)
 * and upload them to the current CUDA device.  The descriptor and all arrays
 * it points to are host memory owned by the caller and are deep-copied; the
 * caller may free them on return.  *out receives a handle owned by the
 * caller, released with robast_free_geometry.  Synchronous.
 * Errors: ROBAST_E_NULL, ROBAST_E_INVALID (message names the surface and
 * field), ROBAST_E_OOM, ROBAST_E_CUDA.
 */
int robast_build_geometry(const robast_geom_desc* desc, robast_geom** out);

/* Free a geometry (NULL is ignored).  Synchronises the device first. */
void robast_free_geometry(robast_geom* g);

/* Geometry facts: number of surfaces, variants, BVH nodes. */
int robast_geometry_info(const robast_geom* g, int32_t* n_surfaces, int32_t* n_variants, int32_t* n_bvh_nodes);

/* ---------------------------------------------------------------- trace */
/*
 * Output arrays (device pointers, caller-owned, n photons).  Any pointer may
 * be NULL, in which case that field is not written.
 *   status [n] u8, bounces [n] u8 (interactions incl. the terminating one),
 *   hit [3n] final position (the detecting / absorbing point, or the last
 *        interaction point, or the origin if there was none),
 *   dir [3n] final direction, last_surface [n] i32 (-1: none),
 *   focal_xy [2n] local (x, y) on the focal surface (DETECTED only, else 0),
 *   counters [ROBAST_N_COUNTERS] u64, atomically accumulated,
 *   err [2n] f32, FP32 trace only: per photon, the running first-order estimate of
 *        the rounding error of the final position (m, row 0) and direction (rad,
 *        row 1) against an exact trace of the same inputs; -1, -1 where the result
 *        comes from the FP64 re-trace of the accuracy guard (robast_trace_opts),
 *   retraced [2] u64, atomically accumulated: [0] photons of the FP32 trace
 *        re-traced in FP64 by the accuracy guard, [1] photons over the guard's
 *        bounds that did not fit its queue and keep their FP32 result.
 */
typedef struct robast_trace_out {
    uint8_t* status;
    uint8_t* bounces;
    void* hit;
    void* dir;
    int32_t* last_surface;
    void* focal_xy;
    unsigned long long* counters;
    float* err;
    unsigned long long* retraced;
} robast_trace_out;

/*
 * Photon tracks (Fig. 2a of the paper shows simulated tracks through a cone;
 * this records them without rendering).  Every interaction of the photons
 * with index first .. first + count - 1 appends one record: points[4k..4k+3]
 * = interaction point x, y, z and 0 (trace precision), info[4k..4k+3] =
 * photon index, bounce index (0-based), surface id, status after the
 * interaction (0 = still travelling).  Records are appended in no particular
 * order (sort by photon, then bounce); *n_records (device u64, zero it before
 * the call) counts every interaction, records beyond cap are dropped.  All
 * pointers are device pointers.
 */
typedef struct robast_track_opts {
    int64_t first, count, cap;
    void* points;
    int32_t* info;
    unsigned long long* n_records;
} robast_track_opts;

typedef struct robast_trace_opts {
    int32_t precision;        /* 32 (default) or 64 */
    int32_t max_bounces;      /* 1..255; 0 = 100 */
    void* stream;             /* cudaStream_t; NULL = legacy default stream */
    const int32_t* variant_of_photon; /* device [n] or NULL (all variant 0) */
    int64_t first_photon_id;  /* photon i uses random stream id first_photon_id + i */
    double eps;               /* self-intersection epsilon; 0 = 1e-6 L_sys (FP32) / 1e-9 L_sys (FP64) */
    int32_t block_size;       /* 64, 128 or 256 (512 too for the FP32 trace without sources);
                                 0 = library choice (FP32: 512, FP64, source mode and counting
                                 build: 128) */
    int32_t blocks_per_sm;    /* 0 = as many as fit */
    unsigned long long* work_units; /* device [ROBAST_N_UNITS] or NULL; non-NULL runs the
                                       counting build of the kernel (block 128, slower; FP32
                                       only in source mode) and adds the work units below to
                                       it.  robast_trace_grad adds its own three instead:
                                       FP64 interactions of the forward passes, interactions
                                       replayed by the reverse sweeps, dual-number
                                       interactions */
    int32_t coherent_order;   /* 0: library default (on for n >= 65536), 1: on, -1: off.  On, the
                                 photons are first sorted by origin cell so that each warp traces
                                 neighbouring rays; the results are identical either way.  The
                                 sort's scratch (~5n bytes) is stream-ordered, from a memory pool
                                 owned by g that keeps its largest use until robast_free_geometry */
    const robast_track_opts* track; /* host pointer or NULL: record photon tracks */
    int32_t refill_min;       /* 0..32; 0 = library default (24).  A warp takes new photons for its
                                 idle lanes once at least refill_min of its 32 lanes are idle, or all
                                 of its lanes that still have work to do are.  Waiting keeps the
                                 lanes of a warp on the same bounce of neighbouring photons (coherent
                                 traversal) at the cost of idle lanes; 1 refills at once.  The
                                 results do not depend on it */
    double accuracy_pos;      /* FP32 accuracy guard (0 = off), final-position error bound (m), and */
    double accuracy_dir;      /* final-direction error bound (rad); 0 in one = no bound on it.  The FP32
                                 trace keeps each position as a float pair and re-solves every hit
                                 from the approximate hit point (a few ulps of the local scale instead
                                 of the distance travelled), and every photon carries a first-order
                                 estimate of its accumulated rounding error: per interaction the hit
                                 point moves by (lateral offset + segment x direction error) / |cos
                                 incidence| plus local rounding, the normal by the surface's
                                 curvature (a cone wall's local profile curvature) times that, and
                                 the new direction by twice the normal's error (reflection) or by
                                 Snell's derivative (refraction); errors carried along add
                                 linearly, fresh roundings in quadrature.  A photon whose estimate
                                 exceeds 0.9 of a bound, or that ends in ERROR, is re-traced from its
                                 inputs in FP64 (same random streams, same epsilon) by a second
                                 launch on the same stream, whose result replaces the FP32 one.  The
                                 queue has an entry (8 bytes) per photon, from g's memory pool like
                                 the sort's scratch; source-mode traces run in chunks of 2^27 photons,
                                 each followed by its re-trace, with the queue of their sources.  Off
                                 with photon tracks or the counting build */
} robast_trace_opts;

/* Work units counted when opts.work_units is set: ray-box tests, quadric root
 * solves, aspheric Newton iterations, aperture tests, cylinder tests, box
 * tests, Bezier wall tests, reflections, Fresnel/Snell evaluations, roughness
 * perturbations, Philox calls, frame transforms, compensated re-solves of a
 * hit (FP32 trace). */
#define ROBAST_N_UNITS 13

/* Fill opts with the defaults. */
void robast_trace_opts_default(robast_trace_opts* opts);

/*
 * Trace n photons through g (Sec. 2.1 loop): origins [3n], dirs [3n] (unit
 * length), wavelengths [n] nm, all device pointers of the precision's element
 * type.  Random draws come from Philox4x32-10 with key (seed_lo, seed_hi) and
 * counter (id_lo, id_hi, bounce index, 0), id = first_photon_id + i, so the
 * result of every photon is independent of launch shape and scheduling.
 * robast_trace uses the default options (FP32, 100 bounces, default stream).
 * n = 0 is a no-op.  Errors: ROBAST_E_NULL (g, inputs, out), ROBAST_E_INVALID
 * (precision, max_bounces, n < 0, a variant table without variants),
 * ROBAST_E_CUDA (launch failure).
 */
int robast_trace(const robast_geom* g, const void* origins, const void* dirs, const void* wavelengths, int64_t n,
                 uint64_t seed, const robast_trace_out* out);
int robast_trace_ex(const robast_geom* g, const void* origins, const void* dirs, const void* wavelengths,
                    int64_t n, uint64_t seed, const robast_trace_out* out, const robast_trace_opts* opts);

/*
 * The same trace with HOST inputs and outputs: the library copies the inputs
 * to a device staging area owned by g (grown on demand), traces, copies the
 * outputs back and synchronises before returning.  Output pointers in `out`
 * are host pointers here (counters too, added to).  The photons go in chunks
 * (at least 2^20 photons, at most 8) over two streams owned by g, after the
 * work already queued on opts->stream, so that copies overlap tracing; the
 * results equal one robast_trace_ex over all photons.  Pinned host buffers
 * (cudaHostAlloc) let the copies run asynchronously.
 */
int robast_trace_host(robast_geom* g, const void* origins, const void* dirs, const void* wavelengths, int64_t n,
                      uint64_t seed, const robast_trace_out* out, const robast_trace_opts* opts);

/* --------------------------------------------------- batched source groups */
/*
 * Batched study of many optical-system variants (the concentrator comparison
 * of Sec. 3 / Fig. 2b: collection efficiency against incidence angle for many
 * cone designs).  Photons are not passed in: each source group generates its
 * photons on the device, uniform over a hexagon (flats at 0, 60, 120 deg of x,
 * centre `centre`, in the plane z = centre[2]) with one direction and a
 * wavelength uniform in [lam_min, lam_max] nm, and traces them through its
 * variant.  Photons are numbered across groups in group order; photon i
 * (id = first_photon_id + i) draws candidate points from Philox4x32-10 with
 * counter (id_lo, id_hi, k, 1), k = 0, 1, ..., and accepts the first inside
 * the hexagon (x = (2 u0 - 1) a, y = (2 u1 - 1) 2a / sqrt 3, u = (w + 1/2) 2^-32;
 * wavelength from u2 of the accepted draw); the trace then uses stream 0 as
 * in robast_trace.  Generation is FP64 with every operation rounded
 * separately, rounded to the trace precision afterwards.
 */
typedef struct robast_source_group {
    int32_t variant, reserved;
    int64_t n_photons;
    double centre[3];
    double apothem;
    double dir[3]; /* unit */
    double lam_min, lam_max;
} robast_source_group;

typedef struct robast_sources robast_sources; /* opaque device-resident group table */

/* Upload n_groups groups (host array, deep-copied) for geometry g.  Synchronous.  Also
 * allocates, for one chunk of these photons (at most 2^27 photons), the FP32 accuracy guard's
 * re-trace queue (8 bytes per photon) and the chunk's coherent-order scratch (generated origins
 * and the sort's counts, about 13 bytes per photon), so that robast_trace_sources allocates
 * nothing. */
int robast_sources_create(const robast_geom* g, const robast_source_group* groups, int32_t n_groups,
                          robast_sources** out);
void robast_sources_free(robast_sources* s);
int robast_sources_info(const robast_sources* s, int32_t* n_groups, int64_t* n_photons);

/*
 * Trace every photon of `src` in ONE persistent launch (all variants side by
 * side).  group_counts: device [n_groups * ROBAST_N_COUNTERS] u64, added to
 * (per group: [0] bounces, [1..6] photons per status, [7] photons), e.g.
 * collection efficiency = counts[1] / counts[7].  `out` (device arrays of the
 * total photon count, any field NULL) may be NULL.  opts as for
 * robast_trace_ex (variant_of_photon must be NULL).  Asynchronous; issues
 * only memsets and kernel launches on the stream: per chunk of 2^27 photons,
 * the coherent-order sort of the chunk's generated origins (unless
 * opts->coherent_order is -1), the trace launch and, with the FP32 accuracy
 * guard on, the FP64 re-trace launch of the chunk's queued photons.  It can
 * be captured in a CUDA graph once a first call on the device has run
 * outside the capture (the sort's kernels take their shared-memory size
 * then).  Results do not depend on the order.
 */
int robast_trace_sources(const robast_geom* g, const robast_sources* src, uint64_t seed,
                         unsigned long long* group_counts, const robast_trace_out* out,
                         const robast_trace_opts* opts);

/* -------------------------------------------------------------- gradients */
/*
 * Differentiable objectives (an addition to the paper's method, which
 * optimises designs by hand: tolerance and design studies of Sec. 3).
 * Reading: each photon's path is the one robast_trace takes in
 * expected-weight mode -- mirrors always reflect and the photon carries
 * w = product of R(lambda) instead of an absorb draw; Fresnel choices and
 * roughness use the same Philox draws -- and is held fixed while the
 * parameters move (boundary terms of path changes are excluded).
 *   ROBAST_OBJ_MSR: sum w |q - qbar|^2 / W over DETECTED photons, q = local
 *       (x, y) on the focal surface, W = sum w, qbar = sum w q / W;
 *   ROBAST_OBJ_SOFT_CE: (1/N) sum w sigmoid(m / tau) over all photons, m =
 *       apothem - max_k |x . u_k| at the crossing of the photon's last
 *       segment with its variant's hexagonal focal plane (0 if it heads away
 *       or the photon was obscured);
 *   ROBAST_OBJ_CENTROID_X / _Y: sum w q_x / W (resp. q_y) over DETECTED.
 * Parameters: ROBAST_N_PARAM per surface, [0..1] tilt about local x, y
 * (as robast_surface_desc.tilt), [2..9] A1..A8 (SAG mirrors), [10..15]
 * Bezier control points P0r, P0z, P1r, P1z, P2r, P2z (HEXCONE mirrors);
 * every such mirror a path meets gets its derivatives.  With several
 * variants the objective is the sum of the variants' objectives, each over
 * its own photons (a batch of designs evaluated in one launch).
 */
#define ROBAST_OBJ_MSR 0
#define ROBAST_OBJ_SOFT_CE 1
#define ROBAST_OBJ_CENTROID_X 2
#define ROBAST_OBJ_CENTROID_Y 3
#define ROBAST_N_PARAM 16

/* Number of parameters of g (ROBAST_N_PARAM x surfaces); 0 for NULL. */
int robast_param_count(const robast_geom* g);

/* What parameter p = surface * ROBAST_N_PARAM + slot of d_params means. */
typedef struct robast_param_info {
    int32_t surface; /* surface index (the order of robast_geom_desc.surfaces) */
    int32_t variant; /* the surface's variant */
    int32_t slot;    /* 0, 1 tilt about local x, y; 2..9 A1..A8; 10..15 P0r P0z P1r P1z P2r P2z */
    int32_t active;  /* 1 if robast_trace_grad can give it a nonzero derivative: slots 0..9 of
                        SAG mirrors, slots 10..15 of HEXCONE mirrors; 0 otherwise */
} robast_param_info;

/* Fills out[robast_param_count(g)] (HOST array, caller-owned).  0 or
 * ROBAST_E_NULL. */
int robast_param_layout(const robast_geom* g, robast_param_info* out);

/*
 * Objective value (HOST *value) and, if d_params (device, FP64,
 * [robast_param_count]) is not NULL, d_params += d_obj * d value / d param.
 * Inputs as robast_trace_ex (device, the precision's element type).  One
 * launch, an adjoint trace: each photon's path is found (nearest hits in
 * the trace precision, interactions re-solved in FP64), then the derivative
 * of its objective terms with respect to the ray state is carried backwards
 * through its interactions; the state before each interaction is
 * recomputed from the photon's inputs (nothing per bounce is stored) and the
 * interaction is evaluated in dual numbers seeded on that state and on the
 * surface's parameters.  The recomputations and dual numbers run in the
 * trace precision, except that an FP32 trace of a geometry with HEXCONE
 * surfaces runs them in FP64 (grazing Bezier roots); each dual evaluation
 * starts just short of its hit, in axes shifted to the surface's origin.
 * Sums over photons are 128-bit fixed point with integer atomics: repeated
 * calls give identical bits, in any processing order (opts->coherent_order:
 * 1 sorts the photons by origin cell first, scratch from g's pool; the
 * default 0 does so only for geometries with HEXCONE surfaces and n >= 65536,
 * where it was measured faster; -1 never).  info (HOST, 8 doubles, may be
 * NULL; totals over variants): W, sum w q_x, sum w q_y, sum w |q|^2, sum w sigmoid,
 * N_detected, untracked photons (no gradient: a path of more than 64
 * interactions, or a recomputation that no longer met its surface), N
 * (photons with an invalid variant index are skipped).  Synchronises the
 * stream; uses device scratch owned by g.
 */
int robast_trace_grad(robast_geom* g, const void* origins, const void* dirs, const void* wavelengths, int64_t n,
                      uint64_t seed, int32_t objective, double tau, double d_obj, double* value, double* d_params,
                      const robast_trace_opts* opts, double* info);

/* ----------------------------------------------------------- reductions */
/*
 * Spot diagram statistics (Fig. 1 g-i) of the DETECTED photons of each of
 * n_windows windows of a trace output: window w covers photons starts[w] ..
 * starts[w] + counts[w] - 1 (host arrays).  status [ld] and focal_xy [2 ld]
 * are device pointers to the trace output (precision 32: float, 64: double;
 * local x of photon i at focal_xy[i], y at focal_xy[ld + i]).  Per window,
 * results (HOST, 4 doubles per window) = {N_detected, cx, cy, R80}: centroid
 * of focal_xy and R80 = the nearest-rank 80th percentile (sorted index
 * ceil(0.8 N) - 1) of the distance to the centroid; cx, cy, R80 are NaN when
 * nothing is detected.  Deterministic (fixed-order FP64 sums, exact
 * selection).  Synchronises the stream; uses device scratch owned by g.
 * Errors: ROBAST_E_NULL, ROBAST_E_INVALID (window outside [0, ld), precision).
 */
int robast_psf(robast_geom* g, const uint8_t* status, const void* focal_xy, int64_t ld, int32_t n_windows,
               const int64_t* starts, const int64_t* counts, int32_t precision, void* stream, double* results);

/*
 * robast_psf_noalloc: the same statistics as robast_psf (same arguments minus
 * the geometry, same results) for callers that cannot allocate device memory
 * when they need them -- for example code whose device memory is all owned by
 * a caching allocator, or an embedding with a fixed memory budget.  The paper
 * has no counterpart; this is a property of the library, not of the method.
 *
 * It allocates nothing: its scratch is one fixed array of about 6.4 MB in
 * device memory, defined at file scope in the library, which every GPU that
 * loads the library holds until the process exits; its host buffers are
 * static too.  Limit: at most 64 windows per call (ROBAST_E_INVALID beyond).
 * The first call on a device looks up the array's device address with that
 * device current.  Every call on a device shares the array and leaves its
 * contents behind (each call clears what it needs cleared), so calls whose
 * GPU work overlaps race with one another: issue them one at a time.
 * Synchronises the stream several times and reads intermediate results on the
 * host, so it must not be called while the stream is being captured into a
 * CUDA graph.  The R80 is the exact nearest-rank value, as robast_psf's: a
 * rank that falls among many copies of a few nearly equal values is resolved
 * by counting the copies of each value.  ROBAST_E_INVALID if the rank's final
 * bin still spans 4096 or more distinct doubles after 8 rounds of 4096-bin
 * refinement: possible only for FP64 coordinates whose radii about the
 * centroid come within about 1e-29 of the spot's size of zero without being
 * zero (robast_psf has no such limit).
 */
int robast_psf_noalloc(const uint8_t* status, const void* focal_xy, int64_t ld, int32_t n_windows,
                       const int64_t* starts, const int64_t* counts, int32_t precision, void* stream,
                       double* results);

/* ----------------------------------------------------------- measurement */
/*
 * Measurement helper, not part of the method: FP32 (precision 32) or FP64
 * (64) fused-multiply-add throughput of the current device in FLOP/s (one FMA
 * = 2 FLOP), from independent FMA chains on every SM, timed with CUDA events
 * on `stream` (best of 5 after a warm-up).  Synchronous.  This is the
 * denominator of the ALU roofline the benchmark reports.
 */
int robast_measure_alu_peak(int32_t precision, void* stream, double* flops_per_s);

/* Last error message of this host thread ("" if none). */
const char* robast_last_error(void);

/* Library version string. */
const char* robast_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ROBAST_H */
