// Device side of the non-sequential photon trace (Okumura et al., ICRC 2015,
// Sec. 1 and 2.1): for every photon, find the nearest intersection over all
// surfaces of its optical system, apply the surface's role (mirror: reflect
// with reflectivity and roughness; refracting face: Snell + Fresnel; focal
// surface: detect; obscuration: absorb), repeat until the photon terminates.
//
// GB300 design:
//  * one persistent grid (SM count x resident blocks); each warp refills its
//    idle lanes from a global work counter with ONE atomic per refill round,
//    so lanes whose photon ended are reused immediately instead of idling
//    until the longest photon of the warp is done;
//  * the surface records, the BVH and the material tables are staged in
//    shared memory once per block (they are read by every lane at every
//    bounce);
//  * photon state lives in registers; inputs and outputs are SoA so a warp's
//    loads and stores of consecutive photons coalesce;
//  * FP32 form: every intersection is computed in the surface's own local
//    frame (origin rebased to the vertex) so metre-scale coordinates do not
//    swamp millimetre-scale sags; FP64 is used only for the reflectivity
//    threshold (so absorb decisions are identical to the FP64 form) and for
//    the last Newton step of aspheric / Bezier roots at grazing incidence;
//  * Philox4x32-10 counter-based streams keyed by (seed, photon id, bounce)
//    make every photon's result independent of scheduling.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace robast {

// ----------------------------------------------------------------- layout
enum { SHAPE_SAG = 0, SHAPE_CYL = 1, SHAPE_BOX = 2, SHAPE_HEXCONE = 3 };
enum { ROLE_MIRROR = 0, ROLE_REFRACT = 1, ROLE_FOCAL = 2, ROLE_OBSC = 3 };
enum { AP_NONE = 0, AP_CIRCLE = 1, AP_ANNULUS = 2, AP_SECTOR = 3, AP_HEX = 4, AP_RECT = 5 };
enum { ST_DETECTED = 1, ST_ABSORBED = 2, ST_OBSCURED = 3, ST_ESCAPED = 4, ST_MAXB = 5, ST_ERROR = 6 };

// Feature profile of a kernel instantiation: the surface kinds and interactions whose code it
// carries.  A geometry is traced by a profile that covers its features; leaving the others out
// keeps the loop's instruction footprint small (instruction fetch was the kernels' top stall).
enum : unsigned {
    FT_ASPH = 1,       // even-asphere terms (Newton intersections)
    FT_CYL = 2,        // cylinders
    FT_BOX = 4,        // boxes
    FT_CONE = 8,       // hexagonal Bezier cones
    FT_REFR = 16,      // refracting faces
    FT_CONE_CALL = 32, // the cone intersection out of line (not a feature: code placement)
    FT_ALL = 31,
    FT_TELESCOPE = FT_ASPH | FT_CYL | FT_BOX,  // mirrors, masts, camera boxes
    FT_CONCENTRATOR = FT_CONE | FT_REFR,       // cones behind windows
};

// Surface record: REC values of the working precision T.
//   [0..2] origin   [3..11] rows of the (tilted) local frame
//   SAG:     [12] c  [13] 1+k  [14..21] A1..A8  [28] (1.1 r_bound)^2 (Newton seed domain)
//   CYL:     [12] radius [13] length
//   BOX:     [12..14] half extents
//   HEXCONE: [12..14] r power-basis coefficients, [15..17] z coefficients
//   aperture [22..27]: CIRCLE r^2; ANNULUS rmin^2 rmax^2; SECTOR rmin^2 rmax^2 e0x e0y e1x e1y;
//                      HEX apothem; RECT hx hy
//   [29] bound on the surface's principal curvatures over its aperture (the FP32 error estimate)
//   [30..32] FP32 record: the origin's rounding error (origin - float(origin)), so that the
//        origin is the pair [0..2] + [30..32]; FP64 record: 0
//   [33] SAG: bound on the asphere terms' sag over the Newton seed domain, sum |A_i| r_bound^2i
//        (how far the surface can lie from its base quadric)
//   [34..35] SAG: the aperture's inner and outer radius (ANNULUS, SECTOR; CIRCLE: outer)
enum { F_O = 0, F_R = 3, F_C = 12, F_K1 = 13, F_A = 14, F_AP = 22, F_RB2 = 28, F_KAP = 29, F_OL = 30, F_ADEV = 33,
       F_APR = 34, REC = 36 };
// Integer record: x = shape | role << 4 | aperture << 8 | has_asph << 12 | exact_normal << 13
// (a plane in a frame of 0 / +-1 entries), y = material,
// z = medium front, w = medium back.
// Material record (doubles): [0] n, [1..16] lambda, [17..32] R, [33] sigma.
enum { MAT_REC = 34 };
// Medium record (doubles): [0] n_const, [1..3] B, [4..6] C, [7] n_abs,
// [8..23] absorption-table wavelengths, [24..39] absorption lengths.
enum { MED_REC = 40 };

// Work units counted by the counting instantiation (kernel template flag C):
// the per-unit figures that turn them into algorithmic FLOPs are stated with
// the benchmark.
enum {
    U_AABB = 0,      // ray-box slab tests
    U_SAG = 1,       // quadric (sag) root solves
    U_NEWTON = 2,    // aspheric Newton iterations
    U_APERTURE = 3,  // aperture inclusion tests
    U_CYL = 4,       // cylinder tests
    U_BOX = 5,       // box tests
    U_HEXWALL = 6,   // Bezier wall tests (6 per cone)
    U_REFLECT = 7,   // reflections
    U_REFRACT = 8,   // Fresnel + Snell evaluations
    U_ROUGH = 9,     // roughness perturbations (Box-Muller + basis)
    U_PHILOX = 10,   // Philox4x32-10 calls (integer pipe)
    U_REBASE = 11,   // world -> local frame transforms
    U_REFINE = 12,   // compensated re-solves of the hit (FP32 form)
    U_N = 13
};
#define CNT(k)                         \
    do {                               \
        if constexpr (C) cnt[(k)] += 1u; \
    } while (0)

// BVH node (64 bytes): the boxes of BOTH children and their references, so
// that one node load serves the two box tests of a level.  Child k is an
// internal node (n[k] == 0, ref = node index), a leaf (n[k] > 0, prims
// [ref, ref + n)) or empty (n[k] < 0).
struct Node {
    float lo0[3], hi0[3];
    float lo1[3], hi1[3];
    int ref0, ref1;
    int n0, n1;
};

struct Tables {
    const void* surf;  // n_surf * REC values of T
    const int4* surf_i;
    const Node* nodes;  // node 0 of a variant's BVH is its root
    const int* prims;
    const int4* variants;  // (bvh root node or -1, first unbounded index, n unbounded, first surface)
    const int* glob;       // surfaces without a bounding box, per variant
    const double* mats;
    const double* meds;
    const float* mats32;  // the material records rounded to FP32 (the FP32 kernel's reads), followed
                          // (16-byte aligned) by the medium records rounded to FP32: meds32(tb)
    const float* surf32;  // FP64 tables: the FP32 surface records (global memory), for the FP32
                          // screens of the FP64 search; NULL elsewhere
    int n_surf, n_nodes, n_prims, n_var, n_glob, n_mat, n_med, pad;
};

// A source group (batched concentrator study): photons uniform over a hexagon
// of apothem a (bounding rectangle half-sizes a, R = 2a / sqrt 3) centred at c
// in the plane z = c.z, direction dir, wavelength uniform in [lam0, lam1];
// its photons are work indices first .. first + n - 1.
struct SrcGroup {
    double c[3];
    double a, R;
    double dir[3];
    double lam0, lam1;
    long long first, n;
    int variant;
    float a32;  // a rounded to FP32 (the rejection screen)
    float R32;  // R rounded to FP32
    int pad;
};

// T: arithmetic precision of the trace; IO: element type of the caller's input and output
// arrays (the FP64 re-trace of FP32 photons reads and writes the FP32 arrays).
template <typename T, typename IO = T>
struct TraceArgs {
    Tables tab;
    const IO* o;
    const IO* d;
    const IO* lam;
    const int* vop;
    const int* order;  // optional processing order: work index -> photon index
    long long n;       // photons: the stride of the SoA arrays
    long long n_work;  // work items (n, a chunk of it, or the capacity of a re-trace queue)
    long long work_base;  // first work index of this launch (chunked source-mode launches)
    const unsigned long long* n_work_dev;  // if set: work items = min(*n_work_dev, n_work)
    const long long* queue_in;             // if set: work index -> photon index (FP64 re-trace)
    unsigned long long seed;
    long long first_id;
    int max_bounces;
    int stage;       // stage tables in shared memory
    int refill_min;  // a warp refills when this many lanes are idle (or all of its live lanes are)
    T eps;
    T newton_tol;
    double newton_tol64;
    uint8_t* st;
    uint8_t* nb;
    IO* hit;
    IO* dir;
    int* last;
    IO* fxy;
    unsigned long long* counters;
    unsigned long long* work;
    unsigned long long* units;  // [U_N], counting instantiation only
    const SrcGroup* groups;     // source mode: photons generated on the device
    int n_groups;
    // photon tracks: every interaction of photons tr_first .. tr_first + tr_count - 1
    long long tr_first, tr_count, tr_cap;
    IO* tr_pts;                     // [tr_cap * 4]: x, y, z, 0
    int* tr_info;                   // [tr_cap * 4]: photon, bounce, surface, status after
    unsigned long long* tr_n;       // records appended (may exceed tr_cap)
    unsigned long long* gcounts;  // source mode: [n_groups][8] counters per group
    // FP32 accuracy guard: a photon whose running error estimate exceeds acc_pos (final
    // position, m) or acc_dir (final direction, rad), or that ends in ERROR, is appended to
    // queue_out and re-traced in FP64 by a second launch (queue_in, n_work_dev = queue_n)
    float acc_pos, acc_dir;
    long long* queue_out;
    unsigned long long* queue_n;    // entries appended (may exceed queue_cap)
    long long queue_cap;
    float* err;                     // [2n] per photon: position and direction error estimate
                                    // (-1, -1: the result comes from the FP64 re-trace)
    unsigned long long* retraced;   // [2]: photons re-traced in FP64; photons over a bound that
                                    // did not fit the queue (they keep the FP32 result)
};



// ------------------------------------------------------------ math helpers
__device__ __forceinline__ float t_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double t_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float t_abs(float x) { return fabsf(x); }
__device__ __forceinline__ double t_abs(double x) { return fabs(x); }
__device__ __forceinline__ float t_min(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double t_min(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float t_max(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double t_max(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float t_log(float x) { return logf(x); }
__device__ __forceinline__ double t_log(double x) { return log(x); }
__device__ __forceinline__ void t_sincospi(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void t_sincospi(double x, double* s, double* c) { sincospi(x, s, c); }
__device__ __forceinline__ bool t_finite(float x) { return isfinite(x); }
__device__ __forceinline__ bool t_finite(double x) { return isfinite(x); }
template <typename T> __device__ __forceinline__ T t_inf();
template <> __device__ __forceinline__ float t_inf<float>() { return __int_as_float(0x7f800000); }
template <> __device__ __forceinline__ double t_inf<double>() { return __longlong_as_double(0x7ff0000000000000ll); }

template <typename T>
struct V3 {
    T x, y, z;
};
template <typename T> __device__ __forceinline__ V3<T> mk(T x, T y, T z) { return V3<T>{x, y, z}; }
template <typename T> __device__ __forceinline__ V3<T> operator+(V3<T> a, V3<T> b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
template <typename T> __device__ __forceinline__ V3<T> operator-(V3<T> a, V3<T> b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
template <typename T> __device__ __forceinline__ V3<T> operator*(T s, V3<T> a) { return mk(s * a.x, s * a.y, s * a.z); }
template <typename T> __device__ __forceinline__ T dot(V3<T> a, V3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename T> __device__ __forceinline__ V3<T> unit(V3<T> a) { return (T(1) / t_sqrt(dot(a, a))) * a; }

// --------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64-bit products, key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

template <typename T>
__device__ __forceinline__ T unit_open(uint32_t w) {
    return (T(w) + T(0.5)) * T(2.3283064365386963e-10);  // 2^-32
}

// Photon of work index idx from its source group (Philox stream 1): rejection
// sampling in the bounding rectangle, candidate k from counter
// (id_lo, id_hi, k, 1).  FP64 with every operation rounded separately, so the
// generated inputs are bit-identical to the CPU reference's.  Returns false if
// 64 candidates were all rejected (probability 0.25^64).
// The candidate (x, y) of draw w in FP64 with every rounding explicit (the definition).
__device__ __forceinline__ void src_xy(const SrcGroup& G, uint4 w, double* x, double* y) {
    const double u0 = __dmul_rn(__dadd_rn((double)w.x, 0.5), 2.3283064365386963e-10);
    const double u1 = __dmul_rn(__dadd_rn((double)w.y, 0.5), 2.3283064365386963e-10);
    *x = __dmul_rn(__dsub_rn(__dmul_rn(2.0, u0), 1.0), G.a);
    *y = __dmul_rn(__dsub_rn(__dmul_rn(2.0, u1), 1.0), G.R);
}

// Inside-hexagon test of the candidate in FP64 (the definition).
__device__ __forceinline__ bool src_inside64(const SrcGroup& G, double x, double y) {
    const double s60 = 0.86602540378443864676;
    const double hx = __dmul_rn(0.5, x), sy = __dmul_rn(s60, y);
    const double m = fmax(fabs(x), fmax(fabs(__dadd_rn(hx, sy)), fabs(__dadd_rn(-hx, sy))));
    return m <= G.a;
}

// Photon pid of group G: the first of up to 64 candidates (Philox stream 1, counter
// (pid, k)) inside the hexagon.  Each candidate is screened in FP32: its hexagon measure m is
// within 2e-6 a of the FP64 value (u to 3 FP32 roundings, x and y to 5e-7 a, the sums to
// 1e-6 a), so a screen outside a band of 1e-5 a around a decides as FP64 would; inside the
// band (about one candidate in 10^5) the FP64 test decides.  The accepted candidate's
// coordinates and wavelength are then formed in FP64 exactly as defined, so the photons are
// the same bits as an all-FP64 generator's (FP64 issues at 1/64 of the FP32 rate here, and a
// rejection loop repeats for the whole warp until its last lane accepts).
__device__ __forceinline__ bool gen_source(const SrcGroup& G, long long pid, uint2 key, double o[3], double* lam) {
    const float s60f = 0.86602540378443864676f;
    for (uint32_t k = 0; k < 64; ++k) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)pid, (uint32_t)((unsigned long long)pid >> 32), k, 1u), key);
        const float u0f = ((float)w.x + 0.5f) * 2.3283064365386963e-10f;
        const float u1f = ((float)w.y + 0.5f) * 2.3283064365386963e-10f;
        const float xf = (2.0f * u0f - 1.0f) * G.a32, yf = (2.0f * u1f - 1.0f) * G.R32;
        const float hxf = 0.5f * xf, syf = s60f * yf;
        const float mf = fmaxf(fabsf(xf), fmaxf(fabsf(hxf + syf), fabsf(syf - hxf)));
        bool inside;
        if (mf < G.a32 * (1.0f - 1e-5f))
            inside = true;
        else if (mf > G.a32 * (1.0f + 1e-5f))
            inside = false;
        else {
            double x, y;
            src_xy(G, w, &x, &y);
            inside = src_inside64(G, x, y);
        }
        if (inside) {
            double x, y;
            src_xy(G, w, &x, &y);
            const double u2 = __dmul_rn(__dadd_rn((double)w.z, 0.5), 2.3283064365386963e-10);
            o[0] = __dadd_rn(G.c[0], x);
            o[1] = __dadd_rn(G.c[1], y);
            o[2] = G.c[2];
            *lam = __dadd_rn(G.lam0, __dmul_rn(__dsub_rn(G.lam1, G.lam0), u2));
            return true;
        }
    }
    return false;
}

// ------------------------------------------------------ frame transforms
// The record S is any indexable source of record values: a pointer into the surface table, or
// (gradient pass) an accessor whose values carry derivatives.
template <typename T, typename SR>
__device__ __forceinline__ V3<T> to_local_pt(SR S, V3<T> p) {
    const T qx = p.x - S[F_O], qy = p.y - S[F_O + 1], qz = p.z - S[F_O + 2];
    return mk(S[F_R + 0] * qx + S[F_R + 1] * qy + S[F_R + 2] * qz, S[F_R + 3] * qx + S[F_R + 4] * qy + S[F_R + 5] * qz,
              S[F_R + 6] * qx + S[F_R + 7] * qy + S[F_R + 8] * qz);
}
template <typename T, typename SR>
__device__ __forceinline__ V3<T> to_local_vec(SR S, V3<T> q) {
    return mk(S[F_R + 0] * q.x + S[F_R + 1] * q.y + S[F_R + 2] * q.z, S[F_R + 3] * q.x + S[F_R + 4] * q.y + S[F_R + 5] * q.z,
              S[F_R + 6] * q.x + S[F_R + 7] * q.y + S[F_R + 8] * q.z);
}
template <typename T, typename SR>
__device__ __forceinline__ V3<T> to_world_vec(SR S, V3<T> q) {
    return mk(S[F_R + 0] * q.x + S[F_R + 3] * q.y + S[F_R + 6] * q.z, S[F_R + 1] * q.x + S[F_R + 4] * q.y + S[F_R + 7] * q.z,
              S[F_R + 2] * q.x + S[F_R + 5] * q.y + S[F_R + 8] * q.z);
}

// ------------------------------------------------------------- apertures
template <typename T, typename SR>
__device__ __forceinline__ bool aperture_inside(SR S, int ap, T x, T y) {
    const T r2 = x * x + y * y;
    switch (ap) {
        case AP_NONE: return true;
        case AP_CIRCLE: return r2 <= T(S[F_AP]);
        case AP_ANNULUS: return r2 >= T(S[F_AP]) && r2 <= T(S[F_AP + 1]);
        case AP_SECTOR:
            return r2 >= T(S[F_AP]) && r2 <= T(S[F_AP + 1]) && (T(S[F_AP + 2]) * y - T(S[F_AP + 3]) * x) >= T(0) &&
                   (x * T(S[F_AP + 5]) - y * T(S[F_AP + 4])) >= T(0);
        case AP_HEX: {
            const T s60 = T(0.86602540378443864676);
            const T m = t_max(t_abs(x), t_max(t_abs(T(0.5) * x + s60 * y), t_abs(-T(0.5) * x + s60 * y)));
            return m <= T(S[F_AP]);
        }
        case AP_RECT: return t_abs(x) <= T(S[F_AP]) && t_abs(y) <= T(S[F_AP + 1]);
    }
    return false;
}

// The aperture grown by m on every side (a point within m of it passes): the asphere's pre-check.
template <typename T, typename SR>
__device__ __forceinline__ bool aperture_near(SR S, int ap, T x, T y, T m) {
    switch (ap) {
        case AP_NONE: return true;
        case AP_CIRCLE: return t_sqrt(x * x + y * y) <= T(S[F_APR + 1]) + m;
        case AP_ANNULUS: {
            const T r = t_sqrt(x * x + y * y);
            return r >= T(S[F_APR]) - m && r <= T(S[F_APR + 1]) + m;
        }
        case AP_SECTOR: {
            const T r = t_sqrt(x * x + y * y);
            return r >= T(S[F_APR]) - m && r <= T(S[F_APR + 1]) + m &&
                   (T(S[F_AP + 2]) * y - T(S[F_AP + 3]) * x) >= -m && (x * T(S[F_AP + 5]) - y * T(S[F_AP + 4])) >= -m;
        }
        case AP_HEX: {
            const T s60 = T(0.86602540378443864676);
            const T h = t_max(t_abs(x), t_max(t_abs(T(0.5) * x + s60 * y), t_abs(-T(0.5) * x + s60 * y)));
            return h <= T(S[F_AP]) + m;
        }
        case AP_RECT: return t_abs(x) <= T(S[F_AP]) + m && t_abs(y) <= T(S[F_AP + 1]) + m;
    }
    return true;
}

template <typename T>
struct LHit {
    T t;
    V3<T> pl;  // local hit point
    V3<T> nl;  // local front normal (unit)
    T u;       // Bezier parameter of a cone-wall hit
};

// sag z(rho) and dz/drho of the even asphere; false outside the conic's domain
template <typename T, typename SR>
__device__ __forceinline__ bool sag_slope(SR S, T rho, T* z, T* slope) {
    const T c = S[F_C];
    const T arg = T(1) - T(S[F_K1]) * c * c * rho;
    if (arg < T(0)) return false;
    const T sq = t_sqrt(arg);
    T poly = T(0), dpoly = T(0);
#pragma unroll
    for (int i = 8; i >= 1; --i) {  // Horner in rho
        poly = poly * rho + T(S[F_A + i - 1]);
        dpoly = dpoly * rho + T(i) * T(S[F_A + i - 1]);
    }
    *z = c * rho / (T(1) + sq) + poly * rho;
    *slope = c / (T(2) * sq) + dpoly;
    return true;
}

// One Newton step on f(t) = z(t) - sag(rho(t)) in FP64 (the final step of an
// FP32 root at grazing incidence).
template <typename T>
__device__ __forceinline__ bool newton_step_fp64(const T* S, V3<T> p, V3<T> d, T* t) {
    double c = (double)S[F_C], k1 = (double)S[F_K1];
    double tt = (double)*t;
    double x = (double)p.x + tt * (double)d.x, y = (double)p.y + tt * (double)d.y, z = (double)p.z + tt * (double)d.z;
    double rho = x * x + y * y;
    double arg = 1.0 - k1 * c * c * rho;
    if (arg < 0.0) return false;
    double sq = sqrt(arg);
    double poly = 0.0, dpoly = 0.0;
#pragma unroll
    for (int i = 8; i >= 1; --i) {
        poly = poly * rho + (double)S[F_A + i - 1];
        dpoly = dpoly * rho + (double)i * (double)S[F_A + i - 1];
    }
    double zs = c * rho / (1.0 + sq) + poly * rho;
    double slope = c / (2.0 * sq) + dpoly;
    double fp = (double)d.z - slope * 2.0 * (x * (double)d.x + y * (double)d.y);
    if (fp == 0.0) return false;
    *t = (T)(tt - (z - zs) / fp);
    return true;
}

// Ray vs SAG surface (local frame).  Quadric F = c (x^2 + y^2 + (1+k) z^2) - 2z,
// sag branch (1+k) c z <= 1; both roots in ascending order, first valid one.
// FP32 screen of an FP64 sag test (no asphere): false if the surface certainly gives no hit.
// It decides only where the FP32 solve is well conditioned: a, b, g and the discriminant each
// lose at most a factor 100 to cancellation, so the roots carry a relative error below 1e-4;
// a root counts as excluded only when it lies more than 1e-3 of the coordinates outside
// [eps, tmax], off the conic's branch, or outside the aperture.
template <typename SR>
__device__ __forceinline__ bool screen_sag_miss(SR S, int ap, V3<float> p, V3<float> d, double eps, double tmax) {
    const float c = (float)S[F_C], k1 = (float)S[F_K1];
    const float px = (float)p.x, py = (float)p.y, pz = (float)p.z;
    const float dx = (float)d.x, dy = (float)d.y, dz = (float)d.z;
    const float ac = fabsf(c), ak = fabsf(k1);
    const float mp = fabsf(px) + fabsf(py) + fabsf(pz);
    const float tm = fminf((float)tmax, 3.0e38f);
    if (c == 0.0f) {  // a plane: t = -pz / dz
        if (!(fabsf(dz) > 1e-2f * (fabsf(dx) + fabsf(dy)))) return true;
        const float t = -pz / dz;
        const float mt = 1e-3f * (fabsf(t) + mp);
        if (!(t > (float)eps - mt) || !(t < tm + mt)) return false;
        const float qx = px + t * dx, qy = py + t * dy;
        return aperture_near(S, ap, qx, qy, mt + 1e-3f * (fabsf(qx) + fabsf(qy)));
    }
    const float a = c * (dx * dx + dy * dy + k1 * dz * dz);
    const float b = c * (px * dx + py * dy + k1 * pz * dz) - dz;
    const float g = c * (px * px + py * py + k1 * pz * pz) - 2.0f * pz;
    const float aa = ac * (dx * dx + dy * dy + ak * dz * dz);
    const float bb = ac * (fabsf(px * dx) + fabsf(py * dy) + ak * fabsf(pz * dz)) + fabsf(dz);
    const float gg = ac * (px * px + py * py + ak * pz * pz) + 2.0f * fabsf(pz);
    if (!(fabsf(a) > 1e-2f * aa) || !(fabsf(b) > 1e-2f * bb) || !(fabsf(g) > 1e-2f * gg)) return true;
    const float disc = b * b - a * g;
    if (!(fabsf(disc) > 1e-2f * (b * b + fabsf(a * g)))) return true;  // FP64 decides
    if (disc < 0.0f) return false;                                      // no root
    const float sq = sqrtf(disc);
    const float qq = -(b + copysignf(sq, b));
    const float r[2] = {qq / a, g / qq};
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float t = r[i];
        const float mt = 1e-3f * (fabsf(t) + mp);
        if (!(t > (float)eps - mt) || !(t < tm + mt)) continue;
        const float qx = px + t * dx, qy = py + t * dy, qz = pz + t * dz;
        if (k1 * c * qz - 1.0f > 1e-2f + ac * ak * mt) continue;  // off the branch (with the point's error)
        if (!aperture_near(S, ap, qx, qy, mt + 1e-3f * (fabsf(qx) + fabsf(qy)))) continue;
        return true;  // a root may hit: FP64 decides
    }
    return false;
}

// FP32 screen of an FP64 aspheric sag test: false only where the FP64 test certainly gives up on
// the surface before its Newton iteration.  The FP64 test takes the first conic root (ascending)
// that lies on the branch and beyond eps; it gives up when that root's point lies outside the
// Newton seed domain or, away from grazing incidence, further outside the aperture than the
// asphere terms can move the hit; and it finds nothing when no root qualifies.  The screen takes
// the same steps on the FP32 solve (well conditioned as in screen_sag_miss: roots to 1e-4
// relative, points to 1e-3 of the coordinates) and decides each comparison only outside that
// margin; anything closer, and any root the FP64 test would hand to Newton, goes to FP64.
template <typename SR>
__device__ __forceinline__ bool screen_asph_miss(SR S, int ap, V3<float> p, V3<float> d, double eps) {
    const float c = (float)S[F_C], k1 = (float)S[F_K1];
    if (c == 0.0f) return true;  // a plane base: FP64 decides
    const float px = p.x, py = p.y, pz = p.z, dx = d.x, dy = d.y, dz = d.z;
    const float ac = fabsf(c), ak = fabsf(k1);
    const float mp = fabsf(px) + fabsf(py) + fabsf(pz);
    const float a = c * (dx * dx + dy * dy + k1 * dz * dz);
    const float b = c * (px * dx + py * dy + k1 * pz * dz) - dz;
    const float g = c * (px * px + py * py + k1 * pz * pz) - 2.0f * pz;
    const float aa = ac * (dx * dx + dy * dy + ak * dz * dz);
    const float bb = ac * (fabsf(px * dx) + fabsf(py * dy) + ak * fabsf(pz * dz)) + fabsf(dz);
    const float gg = ac * (px * px + py * py + ak * pz * pz) + 2.0f * fabsf(pz);
    if (!(fabsf(a) > 1e-2f * aa) || !(fabsf(b) > 1e-2f * bb) || !(fabsf(g) > 1e-2f * gg)) return true;
    const float disc = b * b - a * g;
    if (!(fabsf(disc) > 1e-2f * (b * b + fabsf(a * g)))) return true;
    if (disc < 0.0f) return false;  // no conic root: FP64 finds none either
    const float sq = sqrtf(disc);
    const float qq = -(b + copysignf(sq, b));
    const float t1 = qq / a, t2 = g / qq;
    const float tl = fminf(t1, t2), th = fmaxf(t1, t2);
    if (!(th - tl > 2e-3f * (fabsf(tl) + fabsf(th) + mp))) return true;  // their order is uncertain
    const float ep = (float)eps;
#pragma unroll 1
    for (int i = 0; i < 2; ++i) {
        const float t = i ? th : tl;
        const float mt = 1e-3f * (fabsf(t) + mp);
        const float qx = px + t * dx, qy = py + t * dy, qz = pz + t * dz;
        const float v = k1 * c * qz - 1.0f, mv = 1e-2f + ac * ak * mt;
        if (v > mv) continue;             // off the branch in FP64 too
        if (!(v < -mv)) return true;      // on the edge of the branch
        if (t < ep - mt) continue;        // at or before eps in FP64 too
        if (!(t > ep + mt)) return true;  // near eps
        // the first qualifying root: the seed domain, then the pre-check
        const float eq = mt + 1e-3f * (fabsf(qx) + fabsf(qy));
        const float r = sqrtf(qx * qx + qy * qy), rb = sqrtf((float)S[F_RB2]);
        if (r > rb * 1.001f + eq) return false;
        if (!(r < rb * 0.999f - eq)) return true;
        const float mx = -c * qx, my = -c * qy, mz = 1.0f - c * k1 * qz;
        const float nn = mx * mx + my * my + mz * mz;
        const float dn = fabsf(dx * mx + dy * my + dz * mz);
        if (!(dn * dn > 0.0025f * 1.01f * nn)) return true;  // grazing, or near the threshold: Newton in FP64
        const float m = 2.0f * (float)S[F_ADEV] * sqrtf(nn) / dn + 1e-4f * (fabsf(qx) + fabsf(qy) + fabsf(t));
        return aperture_near(S, ap, qx, qy, 1.001f * m + eq);
    }
    return false;  // no root qualifies: FP64 finds no hit
}

// Aspheres: Newton from the first on-branch root beyond eps.
template <bool C, bool ASPH = true, typename T, typename SR>
__device__ __forceinline__ bool hit_sag(SR S, int ap, bool asph, V3<T> p, V3<T> d, T eps, T tmax, T tol, LHit<T>& h,
                                        bool& err, unsigned* cnt) {
    if constexpr (!ASPH) asph = false;  // a profile without aspheres carries no Newton code
    CNT(U_SAG);
    const T c = S[F_C], k1 = S[F_K1];
    const T a = c * (d.x * d.x + d.y * d.y + k1 * d.z * d.z);
    const T b = c * (p.x * d.x + p.y * d.y + k1 * p.z * d.z) - d.z;
    const T g = c * (p.x * p.x + p.y * p.y + k1 * p.z * p.z) - T(2) * p.z;
    T r[2];
    int nr = 0;
    if (a == T(0)) {
        if (b != T(0)) r[nr++] = -g / (T(2) * b);
    } else {
        const T disc = b * b - a * g;
        if (disc >= T(0)) {
            const T sq = t_sqrt(disc);
            const T q = -(b + (b >= T(0) ? sq : -sq));
            if (q != T(0)) {
                const T t1 = q / a, t2 = g / q;
                r[0] = t_min(t1, t2);
                r[1] = t_max(t1, t2);
                nr = 2;
            } else {
                r[nr++] = T(0);
            }
        }
    }
    for (int i = 0; i < nr; ++i) {
        T t = r[i];
        const V3<T> q = p + t * d;
        if (k1 * c * q.z > T(1)) continue;
        if (asph) {
            if (t <= eps) continue;
            if (q.x * q.x + q.y * q.y > T(S[F_RB2])) return false;
            if constexpr (sizeof(T) <= 8) {
                // Pre-check before Newton: the asphere's hit lies within dev / cos of the quadric's
                // (dev = the asphere terms' largest sag, cos = the incidence cosine at the quadric
                // root), so a quadric root further than twice that (plus a rounding slack) outside
                // the aperture cannot give a hit inside it; skipped at grazing incidence.
                const T mx = -c * q.x, my = -c * q.y, mz = T(1) - c * k1 * q.z;
                const T nn = mx * mx + my * my + mz * mz;
                const T dn = t_abs(d.x * mx + d.y * my + d.z * mz);
                if (dn * dn > T(0.0025) * nn) {
                    const T m = T(2) * T(S[F_ADEV]) * t_sqrt(nn) / dn +
                                T(1e-4) * (t_abs(q.x) + t_abs(q.y) + t_abs(t));
                    if (!aperture_near(S, ap, q.x, q.y, m)) return false;
                }
            }
            bool conv = false;
            T slope = T(0);
            for (int it = 0; it < 32; ++it) {
                CNT(U_NEWTON);
                const V3<T> x = p + t * d;
                T z;
                if (!sag_slope(S, x.x * x.x + x.y * x.y, &z, &slope)) return false;
                const T fp = d.z - slope * T(2) * (x.x * d.x + x.y * d.y);
                if (fp == T(0)) break;
                const T dt = (x.z - z) / fp;
                t -= dt;
                if (t_abs(dt) < tol) {
                    conv = true;
                    break;
                }
            }
            if (!conv) {
                err = true;
                return false;
            }
            if constexpr (sizeof(T) == 4) {
                // grazing incidence: |d . N| < 0.05 |N| -> last step in FP64
                const V3<T> x = p + t * d;
                const T nx = -T(2) * x.x * slope, ny = -T(2) * x.y * slope;
                const T dn = d.x * nx + d.y * ny + d.z;
                if (dn * dn < T(0.0025) * (nx * nx + ny * ny + T(1))) {
                    if (!newton_step_fp64(S, p, d, &t)) return false;
                }
            }
            if (t <= eps || t > tmax) return false;
            const V3<T> x = p + t * d;
            T z;
            if (!sag_slope(S, x.x * x.x + x.y * x.y, &z, &slope)) return false;
            CNT(U_APERTURE);
            if (!aperture_inside(S, ap, x.x, x.y)) return false;
            h.t = t;
            h.pl = x;
            h.nl = unit(mk(-T(2) * x.x * slope, -T(2) * x.y * slope, T(1)));
            return true;
        }
        if (t <= eps) continue;
        if (t > tmax) return false;  // roots ascending: nothing nearer follows
        CNT(U_APERTURE);
        if (!aperture_inside(S, ap, q.x, q.y)) continue;
        h.t = t;
        h.pl = q;
        h.nl = unit(mk(-c * q.x, -c * q.y, T(1) - c * k1 * q.z));
        return true;
    }
    return false;
}

// Open cylinder x^2 + y^2 = r^2, 0 <= z <= length.  The quadratic is solved
// about the ray's point of closest approach to the axis, t = t0 + s with
// t0 = -(p.d)_xy / |d_xy|^2: there the linear term vanishes and |p_xy|^2 - r^2
// is formed from a point near the cylinder, which keeps FP32 accurate for
// rays that start tens of metres away.
// FP32 screen of an FP64 cylinder test: false if the cylinder certainly gives no hit.  With the
// ray at least ~6 degrees off the axis (|d_xy|^2 >= 1e-2), the FP32 closest approach to the axis
// carries an error below 2e-5 of (|p| + |t0|); the cylinder is rejected only when the ray passes
// more than 1e-3 of that scale outside the radius, or when the whole chord lies more than that
// outside [eps, tmax] or outside 0 <= z <= length.  Anything else goes to the FP64 test.
template <typename SR>
__device__ __forceinline__ bool screen_cyl_miss(SR S, V3<float> p, V3<float> d, double eps, double tmax) {
    const float rad = (float)S[F_C], len = (float)S[F_K1];
    const float px = (float)p.x, py = (float)p.y, pz = (float)p.z;
    const float dx = (float)d.x, dy = (float)d.y, dz = (float)d.z;
    const float a = dx * dx + dy * dy;
    if (!(a >= 1e-2f * (a + dz * dz))) return true;
    const float t0 = -(px * dx + py * dy) / a;
    const float cx = px + t0 * dx, cy = py + t0 * dy;
    const float m = 1e-3f * (fabsf(px) + fabsf(py) + fabsf(pz) + fabsf(t0));
    const float dist = sqrtf(cx * cx + cy * cy);
    if (dist > rad + m) return false;  // the ray passes outside the tube
    const float H = (rad + m) * rsqrtf(a);  // bound on the half chord
    const float tlo = t0 - H, thi = t0 + H;
    const float mt = m + 1e-3f * H;
    if (thi < (float)eps - mt || tlo > fminf((float)tmax, 3.0e38f) + mt) return false;
    const float z0 = pz + tlo * dz, z1 = pz + thi * dz;
    if (fmaxf(z0, z1) < -mt || fminf(z0, z1) > len + mt) return false;
    return true;
}

template <typename T>
__device__ __forceinline__ bool hit_cyl(const T* S, V3<T> p, V3<T> d, T eps, T tmax, LHit<T>& h) {
    const T rad = S[F_C], len = S[F_K1];
    const T a = d.x * d.x + d.y * d.y;
    if (a == T(0)) return false;
    const T t0 = -(p.x * d.x + p.y * d.y) / a;
    const T cx = p.x + t0 * d.x, cy = p.y + t0 * d.y;  // closest approach in the xy plane
    const T g = (cx - rad) * (cx + rad) + cy * cy;     // |c|^2 - r^2
    if (g > T(0)) return false;
    const T sh = t_sqrt(-g / a);
    T r[2] = {t0 - sh, t0 + sh};
    const int nr = 2;
    for (int i = 0; i < nr; ++i) {
        const T t = r[i];
        if (t <= eps) continue;
        if (t > tmax) return false;
        const V3<T> x = p + t * d;
        if (x.z < T(0) || x.z > len) continue;
        h.t = t;
        h.pl = x;
        h.nl = unit(mk(x.x, x.y, T(0)));
        return true;
    }
    return false;
}

template <typename T>
__device__ __forceinline__ bool hit_box(const T* S, V3<T> p, V3<T> d, T eps, T tmax, LHit<T>& h) {
    const T pp[3] = {p.x, p.y, p.z}, dd[3] = {d.x, d.y, d.z};
    T tn = -t_inf<T>(), tf = t_inf<T>();
    int axn = -1, axf = -1;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const T hw = S[F_C + ax];
        if (dd[ax] == T(0)) {
            if (t_abs(pp[ax]) > hw) return false;
            continue;
        }
        const T t1 = (-hw - pp[ax]) / dd[ax], t2 = (hw - pp[ax]) / dd[ax];
        const T lo = t_min(t1, t2), hi = t_max(t1, t2);
        if (lo > tn) {
            tn = lo;
            axn = ax;
        }
        if (hi < tf) {
            tf = hi;
            axf = ax;
        }
    }
    if (tn > tf) return false;
    T t;
    int ax;
    if (tn > eps) {
        t = tn;
        ax = axn;
    } else if (tf > eps) {
        t = tf;
        ax = axf;
    } else {
        return false;
    }
    if (t > tmax) return false;
    h.t = t;
    h.pl = p + t * d;
    const T comp = ax == 0 ? h.pl.x : (ax == 1 ? h.pl.y : h.pl.z);
    const T s = comp >= T(0) ? T(1) : T(-1);
    h.nl = mk(ax == 0 ? s : T(0), ax == 1 ? s : T(0), ax == 2 ? s : T(0));
    return true;
}

// Hexagonal cone with a quadratic-Bezier wall profile (Sec. 2.2; the Winston
// cone is the case whose control points lie on a parabola).  Wall j faces
// u_j = (cos j pi/3, sin j pi/3); in its (q, z) half-plane the ray crosses
// the profile where dz (r(u) - q0) - dq (z(u) - z0) = 0, a quadratic in u.
// Unevaluated float pairs h + l for the compensated FP32 polish of cone roots: products of
// two floats are exact (fma gives the rounding error), sums keep their rounding error in l.
struct FF {
    float h, l;
};
__device__ __forceinline__ FF ff_of(float a) { return FF{a, 0.0f}; }
__device__ __forceinline__ FF ff_mul(float a, float b) {
    const float h = __fmul_rn(a, b);
    return FF{h, __fmaf_rn(a, b, -h)};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
    const float s = __fadd_rn(a.h, b.h);
    const float bp = __fsub_rn(s, a.h);
    const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bp)), __fsub_rn(b.h, bp));
    return FF{s, __fadd_rn(e, __fadd_rn(a.l, b.l))};
}
__device__ __forceinline__ FF ff_sub(FF a, FF b) { return ff_add(a, FF{-b.h, -b.l}); }
__device__ __forceinline__ FF ff_mulf(FF a, float b) {
    FF p = ff_mul(a.h, b);
    p.l = __fmaf_rn(a.l, b, p.l);
    return p;
}
__device__ __forceinline__ FF ff_mul2(FF a, FF b) {
    FF p = ff_mul(a.h, b.h);
    p.l = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l));
    return p;
}

// the value of a real (or of a dual number's value part) rounded to FP32 (no FP64 instruction
// for an FP32 value)
__device__ __forceinline__ float val_f(float x) { return x; }
__device__ __forceinline__ float val_f(double x) { return (float)x; }
template <typename N>
__device__ __forceinline__ float val_f(const N& x) {
    return (float)x.v;
}

// cos and sin of j x 60 degrees, j = 0..5 (a hexagon's face directions)
static __constant__ float k_hex_c32[6] = {1.0f, 0.5f, -0.5f, -1.0f, -0.5f, 0.5f};
static __constant__ float k_hex_s32[6] = {0.0f, 0.86602540378443864676f, 0.86602540378443864676f, 0.0f,
                                          -0.86602540378443864676f, -0.86602540378443864676f};
static __constant__ double k_hex_c64[6] = {1.0, 0.5, -0.5, -1.0, -0.5, 0.5};
static __constant__ double k_hex_s64[6] = {0.0, 0.86602540378443864676, 0.86602540378443864676, 0.0,
                                           -0.86602540378443864676, -0.86602540378443864676};

template <typename T>
__device__ __forceinline__ void hex_dir(int j, T& c, T& s) {
    if constexpr (sizeof(T) == 4) {
        c = k_hex_c32[j];
        s = k_hex_s32[j];
    } else {
        c = T(k_hex_c64[j]);
        s = T(k_hex_s64[j]);
    }
}

// FP32 screen of wall j of an FP64 cone test: false if the wall certainly gives no hit.  It
// decides only where the FP32 solve is well conditioned (A, B, C and the discriminant each lose at
// most a factor 100 to cancellation, the ray is not near the wall's profile plane's normal), and
// then excludes a root only when it lies more than 1e-3 outside [0, 1] in u, or more than 1e-2
// of the coordinates outside [eps, best] or outside the wall's wedge; any other case goes to the
// FP64 solve, so the result is the FP64 one.
template <typename SR>
__device__ __forceinline__ bool screen_wall_miss(SR S, int j, float px, float py, float pz, float dx, float dy,
                                                 float dz, float eps, float best) {
    const float ra0 = (float)S[F_C], ra1 = (float)S[F_C + 1], ra2 = (float)S[F_C + 2];
    const float za0 = (float)S[F_C + 3], za1 = (float)S[F_C + 4], za2 = (float)S[F_C + 5];
    const float cj = k_hex_c32[j], sj = k_hex_s32[j];
    const float q0 = px * cj + py * sj, dq = dx * cj + dy * sj;
    const float den = dq * dq + dz * dz;
    if (!(den > 1e-2f * (dx * dx + dy * dy + dz * dz))) return true;
    const float A = dz * ra2 - dq * za2, Am = fabsf(dz * ra2) + fabsf(dq * za2);
    const float B = dz * ra1 - dq * za1, Bm = fabsf(dz * ra1) + fabsf(dq * za1);
    const float C = dz * (ra0 - q0) - dq * (za0 - pz);
    const float Cm = fabsf(dz) * (fabsf(ra0) + fabsf(q0)) + fabsf(dq) * (fabsf(za0) + fabsf(pz));
    if (!(fabsf(B) > 1e-2f * Bm) || !(fabsf(C) > 1e-2f * Cm)) return true;
    float us[2];
    int nu = 0;
    if (Am == 0.0f) {  // a straight profile: one root (the FP64 test takes -C / B too)
        us[nu++] = -C / B;
    } else {
        if (!(fabsf(A) > 1e-2f * Am)) return true;
        const float disc = B * B - 4.0f * A * C;
        if (!(fabsf(disc) > 1e-2f * (B * B + 4.0f * fabsf(A * C)))) return true;
        if (disc < 0.0f) return false;
        const float sq = sqrtf(disc);
        const float q = -0.5f * (B + copysignf(sq, B));
        us[nu++] = q / A;
        us[nu++] = C / q;
    }
    const float ls = fabsf(px) + fabsf(py) + fabsf(pz) + fabsf(ra0) + fabsf(ra1) + fabsf(ra2) + fabsf(za0) +
                     fabsf(za1) + fabsf(za2);
#pragma unroll 1
    for (int i = 0; i < nu; ++i) {
        const float u = us[i];
        const float mu = 1e-3f * (1.0f + fabsf(u));
        if (u < -mu || u > 1.0f + mu) continue;
        const float R = ra0 + u * (ra1 + u * ra2), Z = za0 + u * (za1 + u * za2);
        const float t = ((R - q0) * dq + (Z - pz) * dz) / den;
        const float mt = 1e-2f * (fabsf(t) + ls);
        if (!(t > eps - mt) || !(t < best + mt)) continue;
        const float xx = px + t * dx, xy = py + t * dy;
        const float qj = xx * cj + xy * sj;
        const float mw = mt + 1e-3f * (fabsf(xx) + fabsf(xy));
        bool out = false;
#pragma unroll
        for (int m = 0; m < 6; ++m)
            if (m != j && xx * k_hex_c32[m] + xy * k_hex_s32[m] > qj + mw) out = true;
        if (!out) return true;  // a root may hit: FP64 decides
    }
    return false;
}

template <typename T, typename SR>
__device__ __forceinline__ bool hit_hexcone(SR S, V3<T> p, V3<T> d, T eps, T tmax, LHit<T>& h) {
    const T ra0 = S[F_C], ra1 = S[F_C + 1], ra2 = S[F_C + 2];
    const T za0 = S[F_C + 3], za1 = S[F_C + 4], za2 = S[F_C + 5];
    // wall j's outward direction (cos, sin of j x 60 degrees) from constant memory: no
    // local-memory array for a loop-dependent j, no registers held
    auto dir = [&](int j, T& c, T& s) { hex_dir(j, c, s); };
    bool found = false;
    T best = tmax;
    int bj = 0;
    T bu = T(0);
    // Wall j can only be hit where the ray is in its 60-degree wedge, which is bounded by
    // the two half-planes x.(u_j - u_{j+-1}) >= 0 shared with the neighbouring walls.  A wall
    // whose wedge the ray cannot reach on [0, tmax] (with a margin far above rounding) is
    // skipped; the in-wedge test at the hit point below is unchanged, so the result is too.
    // margin: 1e-5 of the scale of any point p + t d, t <= best, far above the in-wedge test's rounding
    // The reach test runs in FP32 in every precision (on duals, on their values): its margin,
    // 1e-5 of the coordinates' scale, is far above FP32 rounding, so no wall is skipped that the
    // exact test would reach.
    const float pxf = val_f(p.x), pyf = val_f(p.y), dxf = val_f(d.x), dyf = val_f(d.y);
    const float mg = 1e-5f * (fabsf(pxf) + fabsf(pyf) + fabsf(dxf) + fabsf(dyf) + 1e-30f);
    // the wall and root loops stay rolled: one copy of the wall code keeps the kernel's
    // instruction footprint small (warps of a concentrator trace sit in different code paths)
#pragma unroll 1
    for (int j = 0; j < 6; ++j) {
        T cjj, sjj;
        dir(j, cjj, sjj);
        bool reach = true;
        const float bestf = fminf(val_f(best), 1e30f);
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int m2 = side ? (j + 1) % 6 : (j + 5) % 6;
            const float ex = k_hex_c32[j] - k_hex_c32[m2], ey = k_hex_s32[j] - k_hex_s32[m2];
            const float a = pxf * ex + pyf * ey, b = dxf * ex + dyf * ey;
            // largest a + b t over t in [0, best]: at t = best if b > 0 (best may be +inf)
            const float top = b > 0.0f ? a + b * bestf : a;
            if (top < -mg * (1.0f + bestf)) reach = false;
        }
        if (!reach) continue;
        if constexpr (sizeof(T) == 8) {
            if (!screen_wall_miss(S, j, pxf, pyf, (float)p.z, dxf, dyf, (float)d.z, (float)eps, bestf)) continue;
        }
        const T q0 = p.x * cjj + p.y * sjj, dq = d.x * cjj + d.y * sjj;
        const T den = dq * dq + d.z * d.z;
        if (den == T(0)) continue;
        const T A = d.z * ra2 - dq * za2;
        const T B = d.z * ra1 - dq * za1;
        const T C = d.z * (ra0 - q0) - dq * (za0 - p.z);
        T us[2];
        int nu = 0;
        if (A == T(0)) {
            if (B != T(0)) us[nu++] = -C / B;
        } else {
            const T disc = B * B - T(4) * A * C;
            if (disc >= T(0)) {
                const T sq = t_sqrt(disc);
                const T q = -T(0.5) * (B + (B >= T(0) ? sq : -sq));
                if (q != T(0)) {
                    us[nu++] = q / A;
                    us[nu++] = C / q;
                } else {
                    us[nu++] = -B / (T(2) * A);
                }
            }
        }
#pragma unroll 1
        for (int i = 0; i < nu; ++i) {
            T u = us[i];
            const T gp = T(2) * A * u + B;
            // one Newton polish of the root; in FP32 at grazing (|g'| small) the coefficients
            // and g(u) are evaluated in unevaluated float pairs (exact products by fma, two-sum
            // additions; about 46 bits), which removes the cancellation in C at FP32 issue rate
            bool polished = false;
            if constexpr (sizeof(T) == 4) {
                // only roots that can still land in [0, 1]: the polish moves a root by far less
                // than 0.01 (FP32 root error at a near-double root is ~1e-4 of the scale)
                if (u > T(-0.01) && u < T(1.01) && t_abs(gp) < T(0.05) * (t_abs(B) + t_abs(A) + t_abs(C) + T(1e-30))) {
                    const FF q0f = ff_add(ff_mul(p.x, cjj), ff_mul(p.y, sjj));
                    const FF dqf = ff_add(ff_mul(d.x, cjj), ff_mul(d.y, sjj));
                    const FF Af = ff_sub(ff_mul(d.z, ra2), ff_mulf(dqf, za2));
                    const FF Bf = ff_sub(ff_mul(d.z, ra1), ff_mulf(dqf, za1));
                    const FF Cf = ff_sub(ff_mulf(ff_sub(ff_of(ra0), q0f), d.z), ff_mul2(dqf, ff_sub(ff_of(za0), ff_of(p.z))));
                    const FF gf = ff_add(ff_mulf(ff_add(ff_mulf(Af, u), Bf), u), Cf);
                    const float gpf = 2.0f * Af.h * u + Bf.h;
                    if (gpf != 0.0f) u = u - (gf.h + gf.l) / gpf;
                    polished = true;
                }
            }
            if (!polished && gp != T(0)) u = u - ((A * u + B) * u + C) / gp;
            if (u < T(0) || u > T(1)) continue;
            const T R = ra0 + u * (ra1 + u * ra2);
            const T Z = za0 + u * (za1 + u * za2);
            const T t = ((R - q0) * dq + (Z - p.z) * d.z) / den;
            if (t <= eps || t > best) continue;
            if (found && !(t < best)) continue;
            const V3<T> x = p + t * d;
            bool inwedge = true;
            bool exact = true;
            if constexpr (sizeof(T) == 8) {
                // FP64: an FP32 screen decides unless a neighbour's measure lies within its margin
                // (1e-5 of the coordinates) of wall j's; then the FP64 test below decides
                const float xf = (float)x.x, yf = (float)x.y;
                const float qjf = xf * k_hex_c32[j] + yf * k_hex_s32[j];
                const float mw = 1e-5f * (fabsf(xf) + fabsf(yf)) + 1e-30f;
                exact = false;
#pragma unroll
                for (int m = 0; m < 6; ++m) {
                    if (m == j) continue;
                    const float v = xf * k_hex_c32[m] + yf * k_hex_s32[m];
                    if (v > qjf + mw) inwedge = false;
                    else if (v > qjf - mw) exact = true;
                }
                if (!inwedge) exact = false;
            }
            if (exact) {
                const T qj = x.x * cjj + x.y * sjj;
                inwedge = true;
#pragma unroll
                for (int m = 0; m < 6; ++m) {
                    T cm, sm;
                    hex_dir(m, cm, sm);
                    if (m != j && x.x * cm + x.y * sm > qj) inwedge = false;
                }
            }
            if (!inwedge) continue;
            found = true;
            best = t;
            bj = j;
            bu = u;
            h.pl = x;
        }
    }
    if (!found) return false;
    const T Rp = ra1 + T(2) * ra2 * bu, Zp = za1 + T(2) * za2 * bu;
    T cb, sb;
    dir(bj, cb, sb);
    h.u = bu;
    h.t = best;
    h.nl = unit(mk(-Zp * cb, -Zp * sb, Rp));
    return true;
}

// ------------------------------------------------ compensated FP32 hit refinement
// The FP32 trace keeps each photon's position as an unevaluated pair hi + lo (per component,
// |lo| <= ulp(hi) / 2).  The nearest-hit search runs on hi alone; the surface it picks is then
// re-solved from the approximate hit point itself, whose local coordinates are small, so the
// hit is found to a few ulps of the local scale instead of a few ulps of the distance the
// photon travelled.
__device__ __forceinline__ void pair_advance(float& hi, float& lo, float t, float d) {
    const float pr = __fmul_rn(t, d);
    const float pe = __fmaf_rn(t, d, -pr);  // exact product = pr + pe
    const float s = __fadd_rn(hi, pr);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(pr, bp));
    const float l = __fadd_rn(lo, __fadd_rn(e, pe));
    hi = __fadd_rn(s, l);
    lo = __fsub_rn(l, __fsub_rn(hi, s));
}

// Signed normal curvatures of the quadric c (x^2 + y^2 + k1 z^2) - 2 z = 0 at its point x, against
// the front normal (-c x, -c y, 1 - c k1 z) / |g|: the normal curvature along a unit tangent v is
// c (1 + (k1 - 1) v_z^2) / |g|, and v_z^2 runs over [0, 1 - n_z^2] = [0, c^2 (x^2 + y^2) / |g|^2].
// dk widens the range on both sides (the asphere terms); a 1e-3 relative margin covers the
// rounding of the point.  Returns the range's mid-point km and width kw.
__device__ __forceinline__ void quadric_curvatures(float c, float k1, V3<float> x, float dk, float& km, float& kw) {
    const float cr2 = c * c * (x.x * x.x + x.y * x.y);
    const float gz = fmaf(-c * k1, x.z, 1.0f);
    const float g2 = fmaf(gz, gz, cr2);
    if (!(g2 > 0.0f)) return;  // keeps the default (sign unknown)
    const float ig = rsqrtf(g2);
    const float ka = c * ig, kb = c * fmaf(k1 - 1.0f, __fdividef(cr2, g2), 1.0f) * ig;
    km = 0.5f * (ka + kb);
    kw = fabsf(ka - kb) + 2.0f * dk + 2e-3f * fmaxf(fabsf(ka), fabsf(kb));
}

// Hit of the ray (P + t d), P = the pair (ph, pl) at (or very near) surface S, re-solved in
// S's local frame for the small parameter dt.  Returns false where no root is found near the
// point (a grazing ray the FP32 search only just met); the caller then keeps the search's hit.
// kap: the curvature bound to use at this hit (the profile's local curvature for a cone wall,
// else the surface's bound); km, kw: the mid-point and width of the signed normal curvatures
// at the hit (the default, sign unknown: 0 and 2 kap).
template <unsigned FEAT>
__device__ __forceinline__ bool refine_hit(const float* S, int shape, bool asph, V3<float> ph, V3<float> plo,
                                           V3<float> d, float& dt, V3<float>& xl, V3<float>& nl, float& kap,
                                           float& km, float& kw) {
    kap = S[F_KAP];
    // signed normal curvatures at the hit (positive: the surface bends towards its front side),
    // as the mid-point km and width kw of their range over tangent directions; the default
    // (an unknown sign) spans [-kap, kap]
    km = 0.0f;
    kw = 2.0f * kap;
    if constexpr ((FEAT & FT_ASPH) == 0) asph = false;
    if (((FEAT & FT_CYL) == 0 && shape == SHAPE_CYL) || ((FEAT & FT_BOX) == 0 && shape == SHAPE_BOX) ||
        ((FEAT & FT_CONE) == 0 && shape == SHAPE_HEXCONE))
        return false;
    // local origin of the ray: (ph - O_hi) + (plo - O_lo), exact to the rounding of small numbers
    const float qx = __fadd_rn(__fsub_rn(ph.x, S[F_O]), __fsub_rn(plo.x, S[F_OL]));
    const float qy = __fadd_rn(__fsub_rn(ph.y, S[F_O + 1]), __fsub_rn(plo.y, S[F_OL + 1]));
    const float qz = __fadd_rn(__fsub_rn(ph.z, S[F_O + 2]), __fsub_rn(plo.z, S[F_OL + 2]));
    const V3<float> p = to_local_vec(S, mk(qx, qy, qz)), dl = to_local_vec(S, d);
    float t = 0.0f;
    switch (shape) {
        case SHAPE_SAG: {
            const float c = S[F_C], k1 = S[F_K1];
            if (!asph) {
                // the quadric's root nearest 0: g / q in the stable form
                const float a = c * (dl.x * dl.x + dl.y * dl.y + k1 * dl.z * dl.z);
                const float b = c * (p.x * dl.x + p.y * dl.y + k1 * p.z * dl.z) - dl.z;
                const float g = c * (p.x * p.x + p.y * p.y + k1 * p.z * p.z) - 2.0f * p.z;
                const float disc = b * b - a * g;
                if (disc < 0.0f) return false;
                const float q = -(b + copysignf(sqrtf(disc), b));
                if (q == 0.0f) return false;
                t = g / q;
                const V3<float> x = p + t * dl;
                xl = x;
                nl = unit(mk(-c * x.x, -c * x.y, 1.0f - c * k1 * x.z));
                quadric_curvatures(c, k1, x, 0.0f, km, kw);
            } else {
                float slope = 0.0f;
                for (int it = 0; it < 2; ++it) {  // Newton from the point: quadratic convergence
                    const V3<float> x = p + t * dl;
                    float z;
                    if (!sag_slope(S, x.x * x.x + x.y * x.y, &z, &slope)) return false;
                    const float fp = dl.z - slope * 2.0f * (x.x * dl.x + x.y * dl.y);
                    if (fp == 0.0f) return false;
                    t -= (x.z - z) / fp;
                }
                const V3<float> x = p + t * dl;
                const float rho = x.x * x.x + x.y * x.y;
                float z;
                if (!sag_slope(S, rho, &z, &slope)) return false;
                xl = x;
                nl = unit(mk(-2.0f * x.x * slope, -2.0f * x.y * slope, 1.0f));
                // the asphere terms P(r) = sum A_i r^2i add at most max(|P''|, |P'/r|) <= sum 2i(2i-1)|A_i| r^(2i-2)
                // to a normal curvature of the base quadric (the slope factor is at most 1)
                float dk = 0.0f;
#pragma unroll
                for (int i = 8; i >= 1; --i) dk = fmaf(dk, rho, (float)(2 * i * (2 * i - 1)) * fabsf(S[F_A + i - 1]));
                quadric_curvatures(S[F_C], S[F_K1], x, dk, km, kw);
            }
            break;
        }
        case SHAPE_CYL: {
            if constexpr ((FEAT & FT_CYL) != 0) {
                const float rad = S[F_C];
                const float a = dl.x * dl.x + dl.y * dl.y;
                const float b = p.x * dl.x + p.y * dl.y;
                const float g = (p.x - rad) * (p.x + rad) + p.y * p.y;  // |p_xy|^2 - r^2
                const float disc = b * b - a * g;
                if (disc < 0.0f) return false;
                const float q = -(b + copysignf(sqrtf(disc), b));
                if (q == 0.0f) return false;
                t = g / q;
                const V3<float> x = p + t * dl;
                xl = x;
                nl = unit(mk(x.x, x.y, 0.0f));
                break;
            }
            break;
        }
        case SHAPE_BOX: {
            if constexpr ((FEAT & FT_BOX) != 0) {
                // the face the point lies on: the axis where it is furthest out relative to the half extent
                const float r0 = fabsf(p.x) / S[F_C], r1 = fabsf(p.y) / S[F_C + 1], r2 = fabsf(p.z) / S[F_C + 2];
                const int ax = r0 >= r1 ? (r0 >= r2 ? 0 : 2) : (r1 >= r2 ? 1 : 2);
                const float pc = ax == 0 ? p.x : (ax == 1 ? p.y : p.z), dc = ax == 0 ? dl.x : (ax == 1 ? dl.y : dl.z);
                if (dc == 0.0f) return false;
                const float sg = pc >= 0.0f ? 1.0f : -1.0f;
                t = (sg * S[F_C + ax] - pc) / dc;
                xl = p + t * dl;
                nl = mk(ax == 0 ? sg : 0.0f, ax == 1 ? sg : 0.0f, ax == 2 ? sg : 0.0f);
                break;
            }
            break;
        }
        case SHAPE_HEXCONE: {
            if constexpr ((FEAT & FT_CONE) != 0) {
                // the wall whose wedge holds the point, then the profile root nearest the point
                int j = 0;
                float best = -3.0e38f;
                for (int m = 0; m < 6; ++m) {
                    float cm, sm;
                    hex_dir(m, cm, sm);
                    const float v = p.x * cm + p.y * sm;
                    if (v > best) {
                        best = v;
                        j = m;
                    }
                }
                float cj, sj;
                hex_dir(j, cj, sj);
                const float ra0 = S[F_C], ra1 = S[F_C + 1], ra2 = S[F_C + 2];
                const float za0 = S[F_C + 3], za1 = S[F_C + 4], za2 = S[F_C + 5];
                const float q0 = best, dq = dl.x * cj + dl.y * sj;
                const float den = dq * dq + dl.z * dl.z;
                if (den == 0.0f) return false;
                const float A = dl.z * ra2 - dq * za2, B = dl.z * ra1 - dq * za1;
                const float C = dl.z * (ra0 - q0) - dq * (za0 - p.z);
                // candidate roots in u; keep the one whose ray parameter is nearest 0
                float us[2];
                int nu = 0;
                if (A == 0.0f) {
                    if (B != 0.0f) us[nu++] = -C / B;
                } else {
                    const float disc = B * B - 4.0f * A * C;
                    if (disc < 0.0f) return false;
                    const float q = -0.5f * (B + copysignf(sqrtf(disc), B));
                    if (q != 0.0f) {
                        us[nu++] = q / A;
                        us[nu++] = C / q;
                    }
                }
                bool got = false;
                float bu = 0.0f;
                for (int i = 0; i < nu; ++i) {
                    float u = us[i];
                    const float gp = 2.0f * A * u + B;
                    if (gp != 0.0f) u -= ((A * u + B) * u + C) / gp;
                    const float R = ra0 + u * (ra1 + u * ra2), Z = za0 + u * (za1 + u * za2);
                    const float tt = ((R - q0) * dq + (Z - p.z) * dl.z) / den;
                    if (!got || fabsf(tt) < fabsf(t)) {
                        got = true;
                        t = tt;
                        bu = u;
                    }
                }
                if (!got) return false;
                xl = p + t * dl;
                const float Rp = ra1 + 2.0f * ra2 * bu, Zp = za1 + 2.0f * za2 * bu;
                nl = unit(mk(-Zp * cj, -Zp * sj, Rp));
                // the wall is straight across the profile plane: its one curvature is the profile's,
                // (r' z'' - z' r'') / (r'^2 + z'^2)^(3/2) at the hit (signed against the normal
                // (-z', r') of the profile plane), with a margin for the hit's error; the other
                // principal curvature is 0
                const float q2 = Rp * Rp + Zp * Zp;
                const float ks = 1.2f * (Rp * 2.0f * za2 - Zp * 2.0f * ra2) / (q2 * sqrtf(q2));
                kap = fabsf(ks);
                km = 0.5f * ks;
                kw = kap;
                break;
            }
            break;
        }
        default: return false;
    }
    if (!(fabsf(t) < 3.0e38f)) return false;
    dt = t;
    return true;
}

template <typename T>
struct Best {
    T t;
    int sid;
    V3<T> pl;
    V3<T> nl;
    bool err;
};

// The cone intersection out of line: the plain trace kernel sits at its register cap, and
// inlining this rarely-taken path there costs spills on every other path; the source-mode
// kernel (uncapped, the cone studies' hot path) keeps it inline.
template <typename T>
__device__ __noinline__ bool hit_hexcone_call(const T* S, V3<T> p, V3<T> d, T eps, T tmax, LHit<T>* h) {
    return hit_hexcone(S, p, d, eps, tmax, *h);
}

// The FP64 search's photon in FP32 for the FP32 screens: the position as a float pair (hi + lo)
// and the direction.
struct Ray32 {
    V3<float> ph, pl, d;
};

template <bool C, unsigned FEAT = FT_ALL, typename T>
__device__ __forceinline__ void test_surface(const Tables& tb, int sid, V3<T> p, V3<T> d, T eps, T tol, Best<T>& bst,
                                             unsigned* cnt, const Ray32& r32, bool use32) {
    CNT(U_REBASE);
    const T* S = reinterpret_cast<const T*>(tb.surf) + (size_t)sid * REC;
    const int flags = tb.surf_i[sid].x;
    const int shape = flags & 15;
    // FP64 nearest-hit search, sag surfaces and cylinders: an FP32 solve rejects the candidate when
    // it is well conditioned and every root lies clearly outside the surface's reach (off the
    // conic's branch, outside [eps, t_best], outside the aperture or the tube's length; for an
    // asphere, where the FP64 test would give up before Newton); any other case goes to the FP64
    // solve, so the result is the FP64 one.
    // With the FP32 records at hand the screen also rebases in FP32 (the position pair minus the
    // origin pair, a few ulps of the local scale; the margins are 1e-3 of the coordinates), so a
    // rejected candidate costs no FP64 instruction.
    bool screened = false;
    if constexpr (sizeof(T) == 8) {
        const bool sag_plain = shape == SHAPE_SAG && ((flags >> 12) & 1) == 0;
        const bool sag_asph = (FEAT & FT_ASPH) != 0 && shape == SHAPE_SAG && ((flags >> 12) & 1) != 0;
        const bool cyl = (FEAT & FT_CYL) != 0 && shape == SHAPE_CYL;
        if (use32 && (sag_plain || sag_asph || cyl)) {
            const float* S32 = tb.surf32 + (size_t)sid * REC;
            const float qx = __fadd_rn(__fsub_rn(r32.ph.x, S32[F_O]), __fsub_rn(r32.pl.x, S32[F_OL]));
            const float qy = __fadd_rn(__fsub_rn(r32.ph.y, S32[F_O + 1]), __fsub_rn(r32.pl.y, S32[F_OL + 1]));
            const float qz = __fadd_rn(__fsub_rn(r32.ph.z, S32[F_O + 2]), __fsub_rn(r32.pl.z, S32[F_OL + 2]));
            const V3<float> q32 = to_local_vec(S32, mk(qx, qy, qz)), d32 = to_local_vec(S32, r32.d);
            const bool may = sag_plain  ? screen_sag_miss(S32, (flags >> 8) & 15, q32, d32, (double)eps, (double)bst.t)
                             : sag_asph ? screen_asph_miss(S32, (flags >> 8) & 15, q32, d32, (double)eps)
                                        : screen_cyl_miss(S32, q32, d32, (double)eps, (double)bst.t);
            if (!may) return;
            screened = true;
        }
    }
    const V3<T> pl = to_local_pt(S, p), dl = to_local_vec(S, d);
    LHit<T> h;
    bool ok = false, err = false;
    switch (shape) {
        case SHAPE_SAG:
            if constexpr (sizeof(T) == 8) {
                if (!screened && ((flags >> 12) & 1) == 0 &&
                    !screen_sag_miss(S, (flags >> 8) & 15, mk((float)pl.x, (float)pl.y, (float)pl.z),
                                     mk((float)dl.x, (float)dl.y, (float)dl.z), (double)eps, (double)bst.t))
                    break;
            }
            ok = hit_sag<C, (FEAT & FT_ASPH) != 0>(S, (flags >> 8) & 15, (flags >> 12) & 1, pl, dl, eps, bst.t, tol, h,
                                                   err, cnt);
            break;
        case SHAPE_CYL:
            if constexpr ((FEAT & FT_CYL) != 0) {
                CNT(U_CYL);
                if constexpr (sizeof(T) == 8) {
                    if (!screened && !screen_cyl_miss(S, mk((float)pl.x, (float)pl.y, (float)pl.z),
                                                      mk((float)dl.x, (float)dl.y, (float)dl.z), (double)eps,
                                                      (double)bst.t))
                        break;
                }
                ok = hit_cyl(S, pl, dl, eps, bst.t, h);
            }
            break;
        case SHAPE_BOX:
            if constexpr ((FEAT & FT_BOX) != 0) {
                CNT(U_BOX);
                ok = hit_box(S, pl, dl, eps, bst.t, h);
            }
            break;
        case SHAPE_HEXCONE:
            if constexpr ((FEAT & FT_CONE) != 0) {
                if constexpr (C) cnt[U_HEXWALL] += 6u;
                if constexpr ((FEAT & FT_CONE_CALL) == 0)
                    ok = hit_hexcone(S, pl, dl, eps, bst.t, h);
                else
                    ok = hit_hexcone_call(S, pl, dl, eps, bst.t, &h);
            }
            break;
    }
    if (err) bst.err = true;
    // nearest t wins; an exact tie goes to the lower surface id
    if (ok && (h.t < bst.t || (h.t == bst.t && sid < bst.sid))) {
        bst.t = h.t;
        bst.sid = sid;
        bst.pl = h.pl;
        bst.nl = h.nl;
    }
}

// Slab test against a float box: entry distance, or +inf on a miss.
// Conservative boxes make the BVH result equal to a brute-force scan over
// every surface.
// (ox, oy, oz) here are the origin pre-multiplied by the inverse direction,
// so every slab distance is one FMA.
__device__ __forceinline__ float box_entry(const float* lo, const float* hi, float ox, float oy, float oz, float ix,
                                           float iy, float iz, float tmax) {
    const float t0x = fmaf(lo[0], ix, -ox), t1x = fmaf(hi[0], ix, -ox);
    const float t0y = fmaf(lo[1], iy, -oy), t1y = fmaf(hi[1], iy, -oy);
    const float t0z = fmaf(lo[2], iz, -oz), t1z = fmaf(hi[2], iz, -oz);
    const float tn = fmaxf(fmaxf(fminf(t0x, t1x), fminf(t0y, t1y)), fmaxf(fminf(t0z, t1z), 0.0f));
    const float tf = fminf(fminf(fmaxf(t0x, t1x), fmaxf(t0y, t1y)), fminf(fmaxf(t0z, t1z), tmax));
    return tn <= tf ? tn : __int_as_float(0x7f800000);
}

constexpr int STACK = 32;

template <bool C, unsigned FEAT = FT_ALL, typename T>
__device__ __forceinline__ void nearest_hit(const Tables& tb, int var, V3<T> p, V3<T> d, T eps, T tol, Best<T>& bst,
                                            bool& overflow, unsigned* cnt) {
    bst.t = t_inf<T>();
    bst.sid = 0x7fffffff;
    bst.err = false;
    const int4 vr = tb.variants[var];
    Ray32 r32{};
    bool use32 = false;
    if constexpr (sizeof(T) == 8) {
        if (tb.surf32) {
            use32 = true;
            r32.ph = mk((float)p.x, (float)p.y, (float)p.z);
            r32.pl = mk((float)(p.x - (double)r32.ph.x), (float)(p.y - (double)r32.ph.y), (float)(p.z - (double)r32.ph.z));
            r32.d = mk((float)d.x, (float)d.y, (float)d.z);
        }
    }
    for (int k = 0; k < vr.z; ++k) test_surface<C, FEAT>(tb, tb.glob[vr.y + k], p, d, eps, tol, bst, cnt, r32, use32);
    if (vr.x < 0) return;
    // Inverse direction with zero components replaced by +-1e-30, so that the
    // FMA slab form never meets inf - inf (the boxes are padded, so a ray grazing
    // a box face cannot lose a surface that lies strictly inside it).
    auto inv = [](float v) -> float { return 1.0f / (fabsf(v) > 1e-30f ? v : copysignf(1e-30f, v)); };
    const float ix = inv((float)d.x), iy = inv((float)d.y), iz = inv((float)d.z);
    const float ox = (float)p.x * ix, oy = (float)p.y * iy, oz = (float)p.z * iz;
    // while-while traversal: every lane first walks internal nodes until its
    // current item is a leaf (or nothing is left), then every lane with a leaf
    // tests its surfaces; the two code paths do not interleave inside a warp.
    int stack[STACK];  // packed (ref | n << 24)
    float stack_t[STACK];
    int sp = 0;
    // float bound of the current best t, rounded up so that no candidate is lost; updated
    // only when a leaf may have changed the best hit
    float tc;
    auto update_tc = [&]() { tc = bst.t == t_inf<T>() ? 3.0e38f : (float)bst.t * 1.0001f + 1e-30f; };
    update_tc();
    auto pop = [&](int& ref, int& n) {
        ref = -1;
        while (sp > 0) {
            --sp;
            if (stack_t[sp] <= tc) {
                ref = stack[sp] & 0xffffff;
                n = stack[sp] >> 24;
                return;
            }
        }
    };
    int ref = vr.x, n = 0;  // the root is an internal node
    while (true) {
        while (n == 0 && ref >= 0) {
            const Node nd = tb.nodes[ref];  // both children are real (a one-leaf tree repeats its leaf)
            if constexpr (C) cnt[U_AABB] += 2u;
            const float e0 = box_entry(nd.lo0, nd.hi0, ox, oy, oz, ix, iy, iz, tc);
            const float e1 = box_entry(nd.lo1, nd.hi1, ox, oy, oz, ix, iy, iz, tc);
            const bool h0 = e0 < 3.4e38f, h1 = e1 < 3.4e38f;
            if (h0 || h1) {
                // nearer child next; with both hit, the farther one waits with its entry distance
                const bool first0 = h0 && (!h1 || e0 <= e1);
                if (h0 && h1) {
                    if (sp >= STACK) {
                        overflow = true;
                        return;
                    }
                    stack[sp] = first0 ? (nd.ref1 | (nd.n1 << 24)) : (nd.ref0 | (nd.n0 << 24));
                    stack_t[sp] = first0 ? e1 : e0;
                    ++sp;
                }
                ref = first0 ? nd.ref0 : nd.ref1;
                n = first0 ? nd.n0 : nd.n1;
            } else {
                pop(ref, n);
            }
        }
        if (ref < 0) break;
        for (int k = 0; k < n; ++k)
            test_surface<C, FEAT>(tb, tb.prims[ref + k], p, d, eps, tol, bst, cnt, r32, use32);
        update_tc();
        pop(ref, n);
    }
}

// Reflectivity threshold floor(R(lambda) 2^32), R piecewise linear, evaluated
// in FP64 with every operation rounded separately (no contraction) so that the
// absorb decision is the same in both precisions and in the CPU reference.
__device__ __forceinline__ unsigned long long refl_threshold(const double* M, double lam) {
    const int n = (int)M[0];
    const double* L = M + 1;
    const double* R = M + 17;
    double r;
    if (n <= 1 || lam <= L[0]) {
        r = R[0];
    } else if (lam >= L[n - 1]) {
        r = R[n - 1];
    } else {
        int i = 0;
        while (i + 1 < n - 1 && lam >= L[i + 1]) ++i;
        const double frac = __ddiv_rn(__dsub_rn(lam, L[i]), __dsub_rn(L[i + 1], L[i]));
        r = __dadd_rn(R[i], __dmul_rn(__dsub_rn(R[i + 1], R[i]), frac));
    }
    const double thr = floor(__dmul_rn(r, 4294967296.0));
    if (thr <= 0.0) return 0ull;
    return (unsigned long long)thr;
}

// Survive iff w0 < floor(R(lambda) 2^32).  The FP32 form first compares with
// an FP32 estimate of the threshold (cached per photon and material) and
// falls back to the exact FP64 threshold only when the draw lies within the
// estimate's error band (relative 1e-5, probability ~1e-5 per reflection), so
// the decision is exactly the FP64 one at FP32 cost.
// M: the material record rounded to FP32 (no FP64 operation on this path).
__device__ __forceinline__ float refl_estimate32(const float* M, float lam) {
    const int n = (int)M[0];
    const float* L = M + 1;
    const float* R = M + 17;
    if (n <= 1 || lam <= L[0]) return R[0];
    if (lam >= L[n - 1]) return R[n - 1];
    int i = 0;
    while (i + 1 < n - 1 && lam >= L[i + 1]) ++i;
    const float frac = (lam - L[i]) / (L[i + 1] - L[i]);
    return R[i] + (R[i + 1] - R[i]) * frac;
}

template <typename T, typename R>
__device__ __forceinline__ T refr_index(const R* Md, T lam_nm) {
    if (Md[0] > R(0)) return (T)Md[0];
    const T l = lam_nm * T(1e-3);
    const T l2 = l * l;
    T n2 = T(1);
#pragma unroll
    for (int i = 0; i < 3; ++i) n2 += (T)Md[1 + i] * l2 / (l2 - (T)Md[4 + i]);
    return t_sqrt(n2);
}

// the FP32 medium records, which follow the FP32 material records (16-byte aligned)
__device__ __forceinline__ const float* meds32(const Tables& tb) {
    return tb.mats32 + ((size_t)tb.n_mat * MAT_REC + 3) / 4 * 4;
}

// Absorption length at lambda (piecewise linear, clamped); <= 0: no absorption.
template <typename T, typename R>
__device__ __forceinline__ T abs_length(const R* Md, T lam) {
    const int n = (int)Md[7];
    if (n <= 0) return T(-1);
    const R* L = Md + 8;
    const R* A = Md + 24;
    if (n == 1 || lam <= (T)L[0]) return (T)A[0];
    if (lam >= (T)L[n - 1]) return (T)A[n - 1];
    int i = 0;
    while (i + 1 < n - 1 && lam >= (T)L[i + 1]) ++i;
    const T frac = (lam - (T)L[i]) / ((T)L[i + 1] - (T)L[i]);
    return (T)A[i] + ((T)A[i + 1] - (T)A[i]) * frac;
}

template <typename T>
__device__ __forceinline__ T fresnel(T n1, T n2, T ci) {
    const T eta = n1 / n2;
    const T s2 = eta * eta * (T(1) - ci * ci);
    if (s2 >= T(1)) return T(1);
    const T ct = t_sqrt(T(1) - s2);
    const T rs = (n1 * ci - n2 * ct) / (n1 * ci + n2 * ct);
    const T rp = (n2 * ci - n1 * ct) / (n2 * ci + n1 * ct);
    return T(0.5) * (rs * rs + rp * rp);
}

// ------------------------------------------------------------ the kernel
template <typename T>
struct Photon {
    V3<T> p, d;
    T lam;
    long long i;  // local index, -1 = idle
    int var;
    int bounces;
    int mat_cache;
    float refl32;  // FP32 estimate of R(lambda) for mat_cache (FP32 form)
    int last;  // last surface hit, -1: none
    int group; // source mode: group of the photon
    bool bad;  // source mode: no point generated
    unsigned long long thr;
    // FP32 form: first-order estimate of the accumulated rounding error (see trace_kernel)
    V3<T> plo; // FP32 form: low parts of the position pair (p, plo)
    float ep;  // lateral offset of the current ray (m)
    float ed;  // direction (rad)
    float eh;  // last interaction point (m)
    float gp, gd;  // the signed carried pair: lateral (m) and direction (rad) parts
};

// STAGED: the tables fit in shared memory and every table pointer is derived
// from the shared array (so the loads are shared-memory loads); otherwise the
// tables are read from global memory through L1.
// SRC: photons come from source groups generated on the device (batched
// study) instead of caller arrays; per-group counters are accumulated.
// Resident 128-thread blocks per SM the FP32 kernel must fit (a register cap:
// 4 blocks = 128 registers, the most that fits 16 warps per SM without
// spilling); the FP64 form is bound by its FP64 pipe and keeps its registers.
#ifndef ROBAST_TRACE_MIN_BLOCKS
#define ROBAST_TRACE_MIN_BLOCKS 4
#endif
#ifndef ROBAST_TRACE_MIN_BLOCKS_SRC
#define ROBAST_TRACE_MIN_BLOCKS_SRC 1  // source mode: uncapped (swept 1, 3, 4; the 128-register cap spills and runs 25% slower)
#endif
#ifndef ROBAST_TRACE_MIN_BLOCKS_F64
#define ROBAST_TRACE_MIN_BLOCKS_F64 1  // FP64: uncapped
#endif
template <typename T, int BLOCK, bool SRC = false>
struct TraceBounds {
    static constexpr int mb =
        sizeof(T) == 8 ? ROBAST_TRACE_MIN_BLOCKS_F64 : SRC ? ROBAST_TRACE_MIN_BLOCKS_SRC : ROBAST_TRACE_MIN_BLOCKS;
    static constexpr int min_blocks = (mb * 128) / BLOCK > 0 ? (mb * 128) / BLOCK : 1;
};

// Rounding units of the FP32 error estimate, per interaction, in ulps of the hit's coordinate
// scale (the local scale of a refined hit, else the world coordinates plus the segment): KT
// for the frame transform (across and along the ray), KA for the root along the ray (KW for an
// unrefined hit, whose root was solved from far away), KP for the new ray's origin; KN ulps on
// the normal and KD on the new direction (reflection or refraction and normalisation).
constexpr float EST_U = 5.9604645e-08f;  // 2^-24
// The estimate needs no correct rounding: square roots and quotients in their fast forms.
__device__ __forceinline__ float est_sqrt(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }
__device__ __forceinline__ float est_hyp(float a, float b) { return est_sqrt(fmaf(a, a, b * b)); }
constexpr float EST_KT = 1.0f * EST_U, EST_KA = 2.0f * EST_U, EST_KW = 5.0f * EST_U, EST_KP = 0.5f * EST_U,
                EST_KN = 1.0f * EST_U, EST_KD = 1.5f * EST_U;
constexpr float EST_KR2 = 2.5f * EST_U;  // a reflection's fresh direction rounding: hypot(2 KN, KD)

template <typename T, int BLOCK, bool C = false, bool STAGED = true, bool SRC = false, typename IO = T,
          unsigned FEAT = FT_ALL>
__global__ void __launch_bounds__(BLOCK, (TraceBounds<T, BLOCK, SRC>::min_blocks)) trace_kernel(TraceArgs<T, IO> A) {
    // the FP32 form carries a running error estimate; the counting build and FP64 do not
    constexpr bool EST = sizeof(T) == 4 && !C;
    // the plain FP32 kernel keeps the cone intersection out of line (it sits at its register cap)
    constexpr unsigned FH = FEAT | ((!SRC && sizeof(T) == 4) ? (unsigned)FT_CONE_CALL : 0u);
    unsigned cnt[U_N];
    if constexpr (C) {
#pragma unroll
        for (int k = 0; k < U_N; ++k) cnt[k] = 0u;
    }
    extern __shared__ __align__(16) unsigned char smem[];
    Tables tb = A.tab;
    if constexpr (STAGED) {
        // stage every table in shared memory: surfaces, int records, nodes,
        // prims, variants, unbounded lists, materials, media (16-byte chunks)
        unsigned char* s = smem;
        auto stage = [&](const void* src, size_t bytes) -> const void* {
            const int4* from = reinterpret_cast<const int4*>(src);
            int4* to = reinterpret_cast<int4*>(s);
            const size_t n16 = (bytes + 15) / 16;
            for (size_t k = threadIdx.x; k < n16; k += BLOCK) to[k] = from[k];
            const void* r = s;
            s += n16 * 16;
            return r;
        };
        // every count is >= 1 (the host pads empty tables with one entry)
        tb.surf = stage(tb.surf, (size_t)tb.n_surf * REC * sizeof(T));
        tb.surf_i = reinterpret_cast<const int4*>(stage(tb.surf_i, (size_t)tb.n_surf * sizeof(int4)));
        tb.nodes = reinterpret_cast<const Node*>(stage(tb.nodes, (size_t)tb.n_nodes * sizeof(Node)));
        tb.prims = reinterpret_cast<const int*>(stage(tb.prims, (size_t)tb.n_prims * sizeof(int)));
        tb.variants = reinterpret_cast<const int4*>(stage(tb.variants, (size_t)tb.n_var * sizeof(int4)));
        tb.glob = reinterpret_cast<const int*>(stage(tb.glob, (size_t)tb.n_glob * sizeof(int)));
        tb.mats = reinterpret_cast<const double*>(stage(tb.mats, (size_t)tb.n_mat * MAT_REC * sizeof(double)));
        tb.meds = reinterpret_cast<const double*>(stage(tb.meds, (size_t)tb.n_med * MED_REC * sizeof(double)));
        if constexpr (sizeof(T) == 4) {  // the two FP32 copies, adjacent as in global memory
            const size_t b32 = ((size_t)tb.n_mat * MAT_REC * sizeof(float) + 15) / 16 * 16;
            tb.mats32 = reinterpret_cast<const float*>(stage(tb.mats32, b32 + (size_t)tb.n_med * MED_REC * sizeof(float)));
        }
        __syncthreads();
    }
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const uint2 key = make_uint2((uint32_t)A.seed, (uint32_t)(A.seed >> 32));
    const long long n = A.n;
    long long n_work = A.n_work;
    if (A.n_work_dev) {
        const unsigned long long q = *A.n_work_dev;
        if ((long long)q < n_work) n_work = (long long)q;
    }

    Photon<T> ph;
    ph.i = -1;
    bool done = false;
    int cur_g = -1;                // source mode: group whose counts this thread holds
    unsigned int gc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    auto flush_group = [&]() {
        if constexpr (SRC) {
            if (cur_g >= 0)
                for (int k = 0; k < 8; ++k)
                    if (gc[k]) {
                        atomicAdd(A.gcounts + (size_t)cur_g * 8 + k, (unsigned long long)gc[k]);
                        gc[k] = 0;
                    }
        }
    };
    unsigned long long my_bounces = 0;
    unsigned int my_retraced = 0;  // FP64 re-trace: photons finished here
    unsigned int my_status[7] = {0, 0, 0, 0, 0, 0, 0};

    while (true) {
        // refill idle lanes: one atomic per warp per round
        const bool need = ph.i < 0 && !done;
        const unsigned m = __ballot_sync(FULL, need);
        const unsigned live = __ballot_sync(FULL, !done);
        if (m && (m == live || __popc(m) >= A.refill_min)) {
            const int leader = __ffs(m) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(A.work, (unsigned long long)__popc(m));
            base = __shfl_sync(FULL, base, leader);
            if (need) {
                const long long widx = (long long)base + __popc(m & lt_mask);
                if (widx < n_work) {
                    const long long idx = A.queue_in ? A.queue_in[widx]
                                          : A.order  ? A.work_base + (long long)A.order[widx]
                                                     : A.work_base + widx;
                    ph.i = idx;
                    if constexpr (SRC) {
                        // group: the last one whose first index is <= idx
                        int lo = 0, hi = A.n_groups - 1;
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (A.groups[mid].first <= idx)
                                lo = mid;
                            else
                                hi = mid - 1;
                        }
                        const SrcGroup& G = A.groups[lo];
                        double o[3], lam;
                        ph.bad = !gen_source(G, A.first_id + idx, key, o, &lam);
                        // rounded to the precision of the caller's arrays first: the FP64 re-trace of
                        // an FP32 photon starts from the same FP32 inputs as the FP32 trace
                        ph.p = mk((T)(IO)o[0], (T)(IO)o[1], (T)(IO)o[2]);
                        ph.d = mk((T)(IO)G.dir[0], (T)(IO)G.dir[1], (T)(IO)G.dir[2]);
                        ph.lam = (T)(IO)lam;
                        ph.var = G.variant;
                        ph.group = lo;
                    } else {
                        ph.p = mk((T)A.o[idx], (T)A.o[n + idx], (T)A.o[2 * n + idx]);
                        ph.d = mk((T)A.d[idx], (T)A.d[n + idx], (T)A.d[2 * n + idx]);
                        ph.lam = (T)A.lam[idx];
                        ph.var = A.vop ? A.vop[idx] : 0;
                        ph.bad = false;
                    }
                    ph.bounces = 0;
                    ph.mat_cache = -1;
                    ph.last = -1;
                    ph.thr = 0;
                    ph.plo = mk(T(0), T(0), T(0));
                    ph.ep = 0.0f;
                    ph.ed = 0.0f;
                    ph.eh = 0.0f;
                    ph.gp = 0.0f;
                    ph.gd = 0.0f;
                } else {
                    done = true;
                }
            }
        }
        if (__all_sync(FULL, done)) break;
        if (ph.i < 0) continue;

        // ---- one bounce
        int status = 0;
        Best<T> bst;
        bool overflow = false;
        V3<T> fpos = mk(T(0), T(0), T(0));
        const bool bad_var = ph.bad || ph.var < 0 || ph.var >= tb.n_var;  // never index past the variant table
        if (!bad_var)
            nearest_hit<C, FH>(tb, ph.var, ph.p, ph.d, A.eps, A.newton_tol, bst, overflow, cnt);
        if (bad_var || overflow || bst.err) {
            status = ST_ERROR;
        } else if (bst.sid == 0x7fffffff) {
            status = ST_ESCAPED;
        } else {
            const T* S = reinterpret_cast<const T*>(tb.surf) + (size_t)bst.sid * REC;
            const int4 si = tb.surf_i[bst.sid];
            float e_s = 0.0f;     // FP32: coordinate scale of this hit's rounding
            float e_kap = 0.0f;   // FP32: curvature bound at this hit
            float e_km = 0.0f, e_kw = 0.0f;  // FP32: signed normal curvatures at this hit (mid-point, width)
            bool refined = false;  // FP32: hit re-solved from the compensated position
            if constexpr (sizeof(T) == 4) {
                e_s = fmaxf(fabsf(ph.p.x), fmaxf(fabsf(ph.p.y), fabsf(ph.p.z))) +
                      fmaxf(fabsf(S[F_O]), fmaxf(fabsf(S[F_O + 1]), fabsf(S[F_O + 2]))) + bst.t;
                e_kap = S[F_KAP];
                e_kw = 2.0f * e_kap;
                pair_advance(ph.p.x, ph.plo.x, bst.t, ph.d.x);
                pair_advance(ph.p.y, ph.plo.y, bst.t, ph.d.y);
                pair_advance(ph.p.z, ph.plo.z, bst.t, ph.d.z);
                float dt, kap, km, kw;
                V3<float> xl, nl;
                CNT(U_REFINE);
                // accepted only as a correction of the search's own rounding (a grazing ray
                // whose re-solve lands on the other root keeps the search's hit)
                if (refine_hit<FEAT>(S, si.x & 15, (si.x >> 12) & 1, ph.p, ph.plo, ph.d, dt, xl, nl, kap, km, kw) &&
                    fabsf(dt) <= 1e-4f * e_s) {
                    e_kap = kap;
                    e_km = km;
                    e_kw = kw;
                    pair_advance(ph.p.x, ph.plo.x, dt, ph.d.x);
                    pair_advance(ph.p.y, ph.plo.y, dt, ph.d.y);
                    pair_advance(ph.p.z, ph.plo.z, dt, ph.d.z);
                    bst.pl = xl;
                    bst.nl = nl;
                    refined = true;
                    e_s = fmaxf(fabsf(xl.x), fmaxf(fabsf(xl.y), fabsf(xl.z))) + fabsf(dt);
                }
            } else {
                ph.p = ph.p + bst.t * ph.d;
            }
            ph.last = bst.sid;
            // the interaction's four random words (counter: photon id, bounce index); drawn
            // only where they are used (mirrors, refracting faces), the same words either way
            const long long pid = A.first_id + ph.i;
            const uint4 ctr = make_uint4((uint32_t)pid, (uint32_t)((unsigned long long)pid >> 32), (uint32_t)ph.bounces, 0u);
            uint4 w = make_uint4(0u, 0u, 0u, 0u);
            ph.bounces += 1;
            const int role = (si.x >> 4) & 15;
            const V3<T> n = unit(to_world_vec(S, bst.nl));
            const T d_n = dot(ph.d, n);
            const bool front = d_n < T(0);
            // FP32 error estimate, first order.  A ray whose lateral offset is ep and whose
            // direction is off by ed meets the surface (incidence cosine c = |d.n|, after a
            // segment t) at a point off by el = (ep + t ed) / c along the surface, plus the frame
            // transform's rounding KT s / c (s: the coordinate scale of the hit's rounding); the
            // root adds ea = KA s / c along the ray.  The normal there is off by (curvature
            // bound) x (el + ea sin(incidence)), plus its own rounding (none for a plane in an
            // axis-aligned frame, whose normal comes out exact).  The outgoing ray's lateral
            // offset is el times its own cosine plus ea times the sine of the turn (the part of an
            // along-ray shift that is across the new direction) plus the rounding of its origin.
            // Errors carried along the path add linearly (they may be correlated); the fresh
            // roundings of one interaction are independent of them and of each other and add in
            // quadrature.  One carried error is kept signed, as a (lateral, direction) pair
            // (gp, gd) that travels and turns exactly: the lateral offset a curved mirror turns
            // into a direction error (so that a focusing mirror's next segment takes back part
            // of the offset instead of adding to it, see the mirror branch).
            float e_l = 0.0f, e_a = 0.0f, e_c = 1.0f, e_sn = 0.0f, e_ic = 1.0f, e_lat = 0.0f, e_kn = 0.0f;
            if constexpr (EST) {
                e_c = fmaxf(fabsf((float)d_n), 1e-20f);
                e_sn = est_sqrt(1.0f - e_c * e_c);
                e_ic = __fdividef(1.0f, e_c);
                ph.gp = fmaf((float)bst.t, ph.gd, ph.gp);
                e_lat = fmaf((float)bst.t, ph.ed, ph.ep) + fabsf(ph.gp);
                e_l = est_hyp(e_lat * e_ic, EST_KT * e_s * e_ic);
                e_a = (refined ? EST_KA : EST_KW) * e_s * e_ic;
                ph.eh = est_hyp(e_l, e_a);
                e_kn = ((si.x >> 13) & 1) ? 0.0f : EST_KN;
            }
            // one call site for the draw (a front-side mirror hit or a refracting face)
            if ((role == ROLE_MIRROR && front) || ((FEAT & FT_REFR) != 0 && role == ROLE_REFRACT)) {
                w = philox4x32_10(ctr, key);
                CNT(U_PHILOX);
            }
            if (role == ROLE_OBSC) {
                status = ST_OBSCURED;
            } else if (role == ROLE_FOCAL) {
                if (front) {
                    status = ST_DETECTED;
                    fpos = bst.pl;
                } else {
                    status = ST_OBSCURED;
                }
            } else if (role == ROLE_MIRROR) {
                if (!front) {
                    status = ST_OBSCURED;
                } else {
                    const double* M = tb.mats + (size_t)si.y * MAT_REC;
                    bool survive;
                    if constexpr (sizeof(T) == 4) {
                        if (si.y != ph.mat_cache) {
                            ph.refl32 = refl_estimate32(tb.mats32 + (size_t)si.y * MAT_REC, (float)ph.lam);
                            ph.mat_cache = si.y;
                        }
                        const float est = ph.refl32 * 4294967296.0f;
                        const float wf = (float)w.x;
                        if (fabsf(wf - est) > est * 1e-5f + 1024.0f)
                            survive = wf < est;
                        else
                            survive = (unsigned long long)w.x < refl_threshold(M, (double)ph.lam);
                    } else {
                        if (si.y != ph.mat_cache) {
                            ph.thr = refl_threshold(M, (double)ph.lam);
                            ph.mat_cache = si.y;
                        }
                        survive = (unsigned long long)w.x < ph.thr;
                    }
                    if (!survive) {
                        status = ST_ABSORBED;
                    } else {
                        V3<T> nn = n;
                        const T sigma = sizeof(T) == 4 ? (T)tb.mats32[(size_t)si.y * MAT_REC + 33] : (T)M[33];
                        if (sigma > T(0)) {
                            CNT(U_ROUGH);
                            const T u1 = unit_open<T>(w.y), u2 = unit_open<T>(w.z);
                            const T rad = t_sqrt(T(-2) * t_log(u1));
                            T sn, cs;
                            t_sincospi(T(2) * u2, &sn, &cs);
                            const T g1 = rad * cs, g2 = rad * sn;
                            // Duff et al. 2017 orthonormal basis around n
                            const T sgn = n.z >= T(0) ? T(1) : T(-1);
                            const T aa = T(-1) / (sgn + n.z);
                            const T bb = n.x * n.y * aa;
                            const V3<T> tt = mk(T(1) + sgn * n.x * n.x * aa, sgn * bb, -sgn * n.x);
                            const V3<T> bv = mk(bb, sgn + n.y * n.y * aa, -n.y);
                            nn = unit(n + (sigma * g1) * tt + (sigma * g2) * bv);
                        }
                        ph.d = unit(ph.d - (T(2) * dot(ph.d, nn)) * nn);
                        CNT(U_REFLECT);
                        if constexpr (EST) {
                            // A lateral offset L of the incoming ray moves the hit along the
                            // surface and so turns the reflected ray by P L, with P between
                            // 2 kmin c (sagittal) and 2 kmax / c (tangential) for signed normal
                            // curvatures in [kmin, kmax] = km -+ kw / 2.  Their mean over
                            // transverse directions, pm = km (c + 1/c), is applied signed; the
                            // rest, at most pr = |km| (1/c - c) + kw / c, goes to the box.  Of
                            // the two carried laterals (the box's, ep + t ed, and the signed
                            // pair's) the larger becomes the signed pair, turned by -pm; the
                            // other joins the box with its turn.  Fresh: the normal's error from
                            // this hit's own rounding, the normal's and the new direction's
                            // rounding, the outgoing origin's rounding and the part of the
                            // along-ray error across the new direction (sine of the turn 2 s c).
                            const float pm = e_km * (e_c + e_ic);
                            const float pr = fmaf(fabsf(e_km), e_ic - e_c, e_kw * e_ic);
                            const float lb = fmaf((float)bst.t, ph.ed, ph.ep);
                            const float gd1 = fmaf(-pm, ph.gp, ph.gd);
                            float dcar, lcar;
                            if (lb > fabsf(ph.gp)) {
                                dcar = fabsf(gd1);
                                lcar = fabsf(ph.gp);
                                ph.gp = lb;
                                ph.gd = -pm * lb;
                            } else {
                                dcar = fabsf(pm) * lb;
                                lcar = lb;
                                ph.gd = gd1;
                            }
                            const float e_nf = e_kap * fmaf(EST_KT * e_s, e_ic, e_a * e_sn);
                            ph.ed = est_hyp(ph.ed + dcar + pr * e_lat + 2.0f * e_nf, est_hyp(2.0f * e_kn, EST_KD));
                            ph.ep = lcar + est_hyp(fmaf(EST_KT, e_s, e_a * (2.0f * e_sn * e_c)), EST_KP * e_s);
                        }
                    }
                }
            } else if constexpr ((FEAT & FT_REFR) != 0) {  // ROLE_REFRACT: bulk absorption of the segment, then Snell + unpolarised Fresnel
                const int med = front ? si.z : si.w;
                const T len = sizeof(T) == 4 ? abs_length<T>(meds32(tb) + (size_t)med * MED_REC, ph.lam)
                                             : abs_length<T>(tb.meds + (size_t)med * MED_REC, ph.lam);
                if (len > T(0)) {
                    const T surv = (sizeof(T) == 4) ? (T)expf(-(float)(bst.t / len)) : (T)exp(-(double)(bst.t / len));
                    if (!(unit_open<T>(w.w) < surv)) status = ST_ABSORBED;
                }
            }
            if ((FEAT & FT_REFR) != 0 && status == 0 && role == ROLE_REFRACT) {
                T na, nb;
                if constexpr (sizeof(T) == 4) {  // FP32 copy of the medium records: no FP64 instruction
                    na = refr_index<T>(meds32(tb) + (size_t)si.z * MED_REC, ph.lam);
                    nb = refr_index<T>(meds32(tb) + (size_t)si.w * MED_REC, ph.lam);
                } else {
                    na = refr_index<T>(tb.meds + (size_t)si.z * MED_REC, ph.lam);
                    nb = refr_index<T>(tb.meds + (size_t)si.w * MED_REC, ph.lam);
                }
                // the estimate's signed pair joins the box at a refracting face: the face's
                // turn depends on the plane of incidence (no mean to keep signed)
                float e_in = 0.0f, e_nc = 0.0f;
                if constexpr (EST) {
                    e_in = ph.ed + fabsf(ph.gd);
                    ph.gp = 0.0f;
                    ph.gd = 0.0f;
                    e_nc = e_kap * fmaf(e_a, e_sn, e_l);
                }
                const T n1 = front ? na : nb, n2 = front ? nb : na;
                const V3<T> nf = front ? n : T(-1) * n;
                const T ci = -dot(ph.d, nf);
                const T R = fresnel(n1, n2, ci);
                CNT(U_REFRACT);
                if (unit_open<T>(w.x) < R) {
                    ph.d = unit(ph.d - (T(2) * dot(ph.d, nf)) * nf);
                    CNT(U_REFLECT);
                    if constexpr (EST) {
                        // the direction error grows by twice the normal's; the outgoing ray
                        // leaves at the incidence cosine and turns by twice the incidence angle
                        ph.ed = est_hyp(e_in + 2.0f * e_nc, est_hyp(2.0f * e_kn, EST_KD));
                        ph.ep = est_hyp(e_l * e_c + e_a * (2.0f * e_sn * e_c), EST_KP * e_s);
                    }
                } else {
                    const T eta = n1 / n2;
                    const T s2 = eta * eta * (T(1) - ci * ci);
                    const T ct = t_sqrt(T(1) - s2);
                    ph.d = unit(eta * ph.d + (eta * ci - ct) * nf);
                    if constexpr (EST) {
                        // Snell: cos(theta_t) dtheta_t = eta cos(theta_i) dtheta_i, with the angles
                        // measured from a normal that is itself off by e_n; the transmitted ray
                        // leaves at cosine ct and turns by theta_i - theta_t
                        const float ctf = fmaxf((float)ct, 1e-20f);
                        const float g = __fdividef((float)(eta * ci), ctf);
                        const float e_n = est_hyp(e_nc, e_kn);
                        ph.ed = est_hyp((e_in + e_n) * g + e_n, EST_KD);
                        const float st = est_sqrt(1.0f - ctf * ctf);
                        ph.ep = est_hyp(e_l * ctf + e_a * fabsf(e_sn * ctf - e_c * st), EST_KP * e_s);
                    }
                }
            }
            if (status == 0 && !(t_finite(ph.d.x) && t_finite(ph.d.y) && t_finite(ph.d.z))) status = ST_ERROR;
            if (status == 0 && ph.bounces >= A.max_bounces) status = ST_MAXB;
            if (A.tr_pts && ph.i >= A.tr_first && ph.i < A.tr_first + A.tr_count) {
                const unsigned long long k = atomicAdd(A.tr_n, 1ull);
                if ((long long)k < A.tr_cap) {
                    A.tr_pts[4 * k + 0] = (IO)(ph.p.x + ph.plo.x);
                    A.tr_pts[4 * k + 1] = (IO)(ph.p.y + ph.plo.y);
                    A.tr_pts[4 * k + 2] = (IO)(ph.p.z + ph.plo.z);
                    A.tr_pts[4 * k + 3] = IO(0);
                    A.tr_info[4 * k + 0] = (int)ph.i;
                    A.tr_info[4 * k + 1] = ph.bounces - 1;
                    A.tr_info[4 * k + 2] = ph.last;
                    A.tr_info[4 * k + 3] = status;
                }
            }
        }
        if (status == 0) continue;
        // ---- photon finished: store (SoA)
        const long long i = ph.i;
        if constexpr (sizeof(T) == 4) ph.p = ph.p + ph.plo;  // the position pair, rounded
        if constexpr (EST) {
            // the stored position adds its own rounding
            const float e_pos = est_hyp(ph.eh, 0.5f * EST_U * fmaxf(fabsf(ph.p.x), fmaxf(fabsf(ph.p.y), fabsf(ph.p.z))));
            const float e_dir = ph.ed + fabsf(ph.gd);
            if (A.err) {
                A.err[i] = e_pos;
                A.err[n + i] = e_dir;
            }
            // over a bound (or an ERROR, which FP64 may not reproduce): re-traced in FP64 by the
            // next launch, which writes every output and counts the photon
            if (A.queue_out && (e_pos > A.acc_pos || e_dir > A.acc_dir || status == ST_ERROR)) {
                const unsigned long long k = atomicAdd(A.queue_n, 1ull);
                if ((long long)k < A.queue_cap) {
                    A.queue_out[k] = i;
                    ph.i = -1;
                    continue;
                }
                atomicAdd(A.retraced + 1, 1ull);
            }
        } else {
            if (A.queue_in && A.err) {
                A.err[i] = -1.0f;
                A.err[n + i] = -1.0f;
            }
        }
        if (A.st) A.st[i] = (uint8_t)status;
        if (A.nb) A.nb[i] = (uint8_t)ph.bounces;
        if (A.hit) {
            A.hit[i] = (IO)ph.p.x;
            A.hit[n + i] = (IO)ph.p.y;
            A.hit[2 * n + i] = (IO)ph.p.z;
        }
        if (A.dir) {
            A.dir[i] = (IO)ph.d.x;
            A.dir[n + i] = (IO)ph.d.y;
            A.dir[2 * n + i] = (IO)ph.d.z;
        }
        if (A.fxy) {
            A.fxy[i] = (IO)fpos.x;
            A.fxy[n + i] = (IO)fpos.y;
        }
        if (A.last) A.last[i] = ph.last;
        my_bounces += (unsigned long long)ph.bounces;
        if (A.queue_in) ++my_retraced;
        my_status[status] += 1u;
        if constexpr (SRC) {
            if (ph.group != cur_g) {
                flush_group();
                cur_g = ph.group;
            }
            gc[0] += (unsigned)ph.bounces;
            gc[status] += 1u;
            gc[7] += 1u;
        }
        ph.i = -1;
    }
    flush_group();
    if constexpr (C) {
        // per-thread unit counts -> warp sums -> one atomic per warp and unit
#pragma unroll
        for (int k = 0; k < U_N; ++k) {
            const unsigned v = __reduce_add_sync(FULL, cnt[k]);
            if (lane == 0 && v) atomicAdd(A.units + k, (unsigned long long)v);
        }
    }
    if (A.queue_in && A.retraced) {
        const unsigned v = __reduce_add_sync(FULL, my_retraced);
        if (lane == 0 && v) atomicAdd(A.retraced, (unsigned long long)v);
    }
    // warp-aggregated counters
    if (A.counters) {
        unsigned long long b = my_bounces;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) b += __shfl_xor_sync(FULL, b, off);
        unsigned int tot = 0;
        unsigned int sc[7];
#pragma unroll
        for (int k = 1; k < 7; ++k) {
            sc[k] = __reduce_add_sync(FULL, my_status[k]);
            tot += sc[k];
        }
        if (lane == 0) {
            if (b) atomicAdd(A.counters + 0, b);
#pragma unroll
            for (int k = 1; k < 7; ++k)
                if (sc[k]) atomicAdd(A.counters + k, (unsigned long long)sc[k]);
            if (tot) atomicAdd(A.counters + 7, (unsigned long long)tot);
        }
    }
}

}  // namespace robast
