/*
 * FP64 CPU oracle for the non-sequential photon trace (test infrastructure).
 *
 * This header belongs to the oracle alone.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg load the oracle; the product
 * library never does, and the two share no code, header or table.
 *
 * What it computes (Okumura, Noda, Rulten, ICRC 2015, Sec. 2.1-2.2): each
 * photon moves along a straight line until the NEAREST intersection over every
 * surface of its optical system (non-sequential: no surface order is given in
 * advance).  The role of the surface that was hit decides what happens:
 * mirrors reflect, lens faces refract, the focal surface detects, obscurations
 * absorb.  The loop repeats until the photon terminates.  The surface shapes
 * are the primitive shapes used by the paper's telescope models plus the
 * aspheric disk, the Winston cone and the Bezier-profile cone of Sec. 2.2.
 * Everything quantitative the paper leaves open (epsilons, tie-breaks, the
 * reflectivity draw, roughness, Fresnel, random streams) is fixed by the
 * readings listed in the design notes of this repository.
 */
#ifndef ROBAST_ORACLE_H
#define ROBAST_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* shapes */
enum { O_SHAPE_SAG = 0, O_SHAPE_CYLINDER = 1, O_SHAPE_BOX = 2, O_SHAPE_HEXCONE = 3 };
/* roles (Sec. 2.1: AMirror, ALens, AFocalSurface, AObscuration) */
enum { O_ROLE_MIRROR = 0, O_ROLE_REFRACT = 1, O_ROLE_FOCAL = 2, O_ROLE_OBSCURATION = 3 };
/* apertures of a sag surface, tested on the local (x, y) of the hit point */
enum { O_AP_NONE = 0, O_AP_CIRCLE = 1, O_AP_ANNULUS = 2, O_AP_SECTOR = 3, O_AP_HEXAGON = 4, O_AP_RECT = 5 };
/* photon end states */
enum { O_ST_DETECTED = 1, O_ST_ABSORBED = 2, O_ST_OBSCURED = 3, O_ST_ESCAPED = 4,
       O_ST_MAX_BOUNCES = 5, O_ST_ERROR = 6 };

typedef struct {
    int32_t shape, role, aperture, material, medium_front, medium_back, pad;
    double origin[3];   /* world position of the local origin (vertex) */
    double rot[9];      /* row-major; row r = local axis r in world coordinates */
    double tilt[2];     /* extra rotation about local x (tilt[0]) then local y (tilt[1]) */
    double curv, conic; /* sag surface: c = 1/R, k */
    double asph[8];     /* A1..A8 multiplying r^2 .. r^16 */
    double ap[4];       /* aperture parameters */
    double prm[8];      /* shape parameters (cylinder, box, hex cone) */
} o_surface;

typedef struct {
    int32_t n, pad;
    double lam[16];     /* nm, ascending */
    double refl[16];
    double sigma;       /* roughness: Gaussian normal tilt per tangent axis, rad */
} o_material;

typedef struct {
    double n_const;     /* > 0: constant index */
    double B[3], C[3];  /* Sellmeier, lambda in micrometres, C in um^2 */
    int32_t n_abs, pad; /* bulk absorption: 0 = none, else a table of n_abs points */
    double abs_lam[16]; /* nm, ascending */
    double abs_len[16]; /* absorption length (m): survival exp(-s / len) over a path s */
} o_medium;

typedef struct {
    int32_t n_surfaces, n_materials, n_media, n_variants;
    const o_surface* surfaces;
    const o_material* materials;
    const o_medium* media;
    const int32_t* variant_offsets; /* n_variants + 1 entries; NULL = one variant */
} o_scene;

typedef struct {
    uint8_t* status;      /* [n] */
    uint8_t* bounces;     /* [n] */
    double* hit;          /* [3n] SoA: x block, y block, z block */
    double* dir;          /* [3n] SoA */
    int32_t* last_surface;/* [n] */
    double* focal_xy;     /* [2n] SoA: local x block, local y block (DETECTED only) */
    double* edge_margin;  /* [n] optional: min relative aperture margin met on the path */
    double* cond;         /* [n] optional: sum over interactions of 1 / |cos(incidence)| */
} o_outputs;

/* A source group: photons uniform over a hexagon (flats at 0, 60, 120 deg,
 * centre c, apothem a) in the plane z = c[2], all with direction dir, and
 * wavelength uniform in [lam_min, lam_max]; the photons of group g are ids
 * first .. first + n - 1 (plus the call's first_photon_id). */
typedef struct {
    int32_t variant, pad;
    int64_t first, n;
    double c[3];
    double apothem;
    double dir[3];
    double lam_min, lam_max;
} o_source_group;

/* Generate the photons of the groups from Philox stream 1 (rejection sampling,
 * draw k of photon id uses counter (id_lo, id_hi, k, 1)).  Writes origins [3n],
 * dirs [3n], wavelengths [n], variant [n] for n = sum of group sizes.  Returns
 * the number of photons that found no point in 64 draws (they get NaN). */
int64_t oracle_generate_sources(const o_source_group* groups, int32_t n_groups, uint64_t seed,
                                int64_t first_photon_id, double* origins, double* dirs, double* wavelengths,
                                int32_t* variant);

/* ------------------------------------------------------------ gradients
 * Frozen-path objectives (a reading: the paper defines no objective).  A
 * nominal trace in expected-weight mode (mirrors always reflect, the photon
 * carries w = product of R(lambda) instead of an absorb draw) records each
 * photon's surface sequence, distances and reflect/refract decisions; the
 * objective is then evaluated on those paths with the parameters moved by
 * `delta`, re-intersecting the recorded surfaces (apertures ignored, the root
 * nearest the recorded distance), so that it is smooth in the parameters.
 *   objective 0, MSR: detected photons, W = sum w, qbar = sum w q / W,
 *                     MSR = sum w |q - qbar|^2 / W (q = focal-surface x, y);
 *   objective 1, soft CE: (1/N) sum w sigmoid(m / tau), m = apothem - max_k
 *                     |x . u_k| at the crossing of the photon's last segment
 *                     with the plane of its variant's (hexagonal) focal
 *                     surface, 0 if the segment does not head into it or the
 *                     photon was obscured;
 *   objectives 2, 3 (closed-form pins only): the w-weighted centroid of the
 *                     DETECTED photons' focal x (2) or y (3).
 * With several variants the objective is the sum of the variants' objectives,
 * each over its own photons.
 * Parameters: 16 per surface -- [0..1] tilt about local x, y; [2..9] A1..A8
 * (SAG mirrors); [10..15] Bezier control points P0r, P0z, P1r, P1z, P2r, P2z
 * (HEXCONE mirrors).  grad (may be NULL): d objective / d parameter by
 * forward-mode dual numbers along the frozen paths, for every differentiable
 * surface a path meets (a path meeting several is replayed with the slots of
 * four of them at a time). */
#define O_N_PARAM 16
int oracle_objective(const o_scene* scene, int64_t n, const double* origins, const double* dirs,
                     const double* wavelengths, const int32_t* variant_of_photon, uint64_t seed,
                     int64_t first_photon_id, int32_t max_bounces, double eps, int32_t n_threads,
                     int32_t objective, double tau, const double* delta, double* value, double* grad);

/* Photon tracks (Fig. 2a shows simulated tracks): trace photons
 * track_first .. track_first + track_count - 1 of the input and record every
 * interaction -- points [3 per record] and info [4 per record: photon index,
 * bounce index (0-based), surface id, status after the interaction (0 =
 * alive)], in photon then bounce order, at most cap records.  Returns the
 * number of interactions (may exceed cap), or < 0 on bad arguments. */
int64_t oracle_track(const o_scene* scene, int64_t n, const double* origins, const double* dirs,
                     const double* wavelengths, const int32_t* variant_of_photon, uint64_t seed,
                     int64_t first_photon_id, int32_t max_bounces, double eps, int64_t track_first,
                     int64_t track_count, double* points, int32_t* info, int64_t cap);

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11). */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Trace n photons (origins/dirs: [3n] SoA, wavelengths in nm).  Returns 0 or <0 on a bad scene. */
int oracle_trace(const o_scene* scene, int64_t n, const double* origins, const double* dirs,
                 const double* wavelengths, const int32_t* variant_of_photon, uint64_t seed,
                 int64_t first_photon_id, int32_t max_bounces, double eps, int32_t n_threads,
                 const o_outputs* out);

/* Building blocks exposed for the pin tests. */
double oracle_fresnel_unpolarised(double n1, double n2, double cos_i);
double oracle_refractive_index(const o_medium* m, double lambda_nm);
double oracle_absorption_length(const o_medium* m, double lambda_nm);
double oracle_reflectivity(const o_material* m, double lambda_nm);
/* Nearest hit of one ray against one surface, world frame.  Returns 1 on hit. */
int oracle_intersect(const o_surface* s, const double p[3], const double d[3], double eps,
                     double* t, double n_front[3], double local_hit[3]);

#ifdef __cplusplus
}
#endif
#endif
