// Gradient kernel: frozen-path objectives and their derivatives with respect
// to the surface parameters (facet tilts, aspheric coefficients, Bezier
// control points).  The paper defines no objective; the reading implemented
// here (shared with the CPU reference, which implements it independently):
//  * each photon's path is the one the trace takes in expected-weight mode
//    (mirrors always reflect and the photon carries w = product of R(lambda)
//    instead of an absorb draw; refraction/Fresnel decisions and roughness
//    use the trace's Philox draws), held fixed when parameters move;
//  * MSR = sum w |q - qbar|^2 / W over DETECTED photons (q = focal-surface
//    local x, y, W = sum w, qbar = sum w q / W); soft CE = (1/N) sum w
//    sigmoid(m / tau), m = the exit-hexagon margin of the crossing of the
//    photon's last segment with its variant's focal plane.
//
// Adjoint method, per photon:
//  1. forward pass: the path's surfaces come from the trace's nearest-hit
//     search (in the trace precision); each interaction is re-solved in FP64,
//     which gives the state, the weight and the objective terms (the MSR
//     gradient contracts the spot coordinates with their centroid, which
//     cancels, so they need FP64).  Only the surface ids, the segment lengths
//     and the refracting faces' reflect/refract decisions are kept, not the
//     states;
//  2. reverse sweep: the derivative of the photon's objective terms with
//     respect to the ray state (point, direction) is carried backwards
//     through the interactions.  For interaction k the state before it is
//     recomputed by replaying interactions 0 .. k-1 from the photon's inputs
//     (known surfaces, no search), and interaction k is evaluated once in
//     forward-mode dual numbers seeded on that state (6 slots) and on the
//     surface's parameters (up to 10 slots): the state Jacobian carries the
//     adjoint one interaction back, the parameter Jacobian contracted with the
//     adjoint is the photon's gradient for that surface.  Every
//     differentiable surface the path meets gets its share, however many.
//     The replays and dual numbers run in precision R: the trace's (FP32
//     for an FP32 trace) or FP64 where Bezier cone walls need it; each dual
//     evaluation starts just short of its hit, in axes shifted to the
//     surface's origin.
// Sums over photons are 128-bit fixed point (two's complement, 64 fraction
// bits) accumulated with integer atomics, so they do not depend on the order
// in which photons finish: repeated runs give identical bits.
#pragma once
#include "dual.cuh"
#include "launch.h"

namespace robast {

constexpr int GW = 16;        // dual slots: 6 ray-state components, then 10 surface parameters
constexpr int GMAXB = 64;     // interactions a path may have and still be differentiated
// dual numbers of the derivative passes, in the trace precision R
template <typename R>
using DR = Dn<R, GW>;

// ------------------------------------------------------------ fixed point
// a[0] = low word (fraction, 2^-64 units), a[1] = high word (integer part, two's complement).
__device__ __forceinline__ void fx_add(unsigned long long* a, double c) {
    if (!(c != 0.0) || !(fabs(c) < 9.0e18)) return;  // zero, NaN or beyond the format
    const double m = fabs(c);
    const double ip = floor(m);
    unsigned long long hi = (unsigned long long)ip;
    unsigned long long lo = (unsigned long long)((m - ip) * 18446744073709551616.0);  // exact fraction x 2^64
    if (c < 0.0) {
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0ull ? 1ull : 0ull);
    }
    const unsigned long long old = atomicAdd(a, lo);
    atomicAdd(a + 1, hi + (old + lo < old ? 1ull : 0ull));
}
// the same for an FP32 contribution, converted with integer operations only (no FP64
// instruction): |c| = m 2^(E - 150) with the 24-bit significand m, so c 2^64 = m 2^(E - 86),
// truncated toward zero like the FP64 form
__device__ __forceinline__ void fx_add(unsigned long long* a, float c) {
    const unsigned b = __float_as_uint(c);
    const int E = (int)((b >> 23) & 0xffu);
    if (E == 0 || E >= 190) return;  // zero or subnormal (far below 2^-64), or |c| >= 2^63 (inf, NaN too)
    const unsigned long long m = (unsigned long long)((b & 0x7fffffu) | 0x800000u);
    const int sh = E - 86;
    unsigned long long lo, hi;
    if (sh >= 64) {
        lo = 0ull;
        hi = m << (sh - 64);
    } else if (sh > 0) {
        lo = m << sh;
        hi = m >> (64 - sh);
    } else if (sh == 0) {
        lo = m;
        hi = 0ull;
    } else if (sh > -64) {
        lo = m >> (-sh);
        hi = 0ull;
    } else {
        return;
    }
    if (b >> 31) {
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0ull ? 1ull : 0ull);
    }
    if ((lo | hi) == 0ull) return;
    const unsigned long long old = atomicAdd(a, lo);
    atomicAdd(a + 1, hi + (old + lo < old ? 1ull : 0ull));
}
// an integer count n into the sum: n units of 2^64 in the high word
__device__ __forceinline__ void fx_add_count(unsigned long long* a, unsigned long long n) {
    if (n) atomicAdd(a + 1, n);
}
__host__ __device__ __forceinline__ double fx_value(const unsigned long long* a) {
    return (double)(long long)a[1] + (double)a[0] * 5.421010862427522e-20;  // 2^-64
}

// R(lambda), piecewise linear in the material's table (clamped)
__device__ __forceinline__ double refl_value(const double* M, double lam) {
    const int n = (int)M[0];
    const double* L = M + 1;
    const double* R = M + 17;
    if (n <= 1 || lam <= L[0]) return R[0];
    if (lam >= L[n - 1]) return R[n - 1];
    int i = 0;
    while (i + 1 < n - 1 && lam >= L[i + 1]) ++i;
    return R[i] + (R[i + 1] - R[i]) * ((lam - L[i]) / (L[i + 1] - L[i]));
}

// Record accessor of the derivative passes: FP64 record values rounded to R, with derivative
// slots 6.. for the parameters of a differentiable surface (mode 1, SAG mirror: tilt x, y ->
// slots 6, 7 through the frame rows, A1..A8 -> slots 8..15; mode 2, HEXCONE mirror: control
// points P0r, P0z, P1r, P1z, P2r, P2z -> slots 6..11 through the power-basis coefficients of the
// profile).  The surface origin reads as 0: a derivative pass works in world axes shifted to the
// surface's origin (the shift is formed in FP64), so its coordinates are small.
template <typename R>
struct GRec {
    const double* S;
    const double* G;  // d rows / d tilt_x (9), d rows / d tilt_y (9)
    int mode;
    __device__ __forceinline__ DR<R> operator[](int k) const {
        if (k >= F_O && k < F_O + 3) return DR<R>(0.0);
        DR<R> r(S[k]);
        if (mode == 1) {
            if (k >= F_R && k < F_R + 9) {
                r.d[6] = (R)G[k - F_R];
                r.d[7] = (R)G[9 + k - F_R];
            } else if (k >= F_A && k < F_A + 8) {
                r.d[8 + (k - F_A)] = R(1);
            }
        } else if (mode == 2) {
            switch (k) {  // r(u) = ra0 + ra1 u + ra2 u^2 with ra0 = P0r, ra1 = 2 (P1r - P0r), ra2 = P0r - 2 P1r + P2r
                case F_C + 0: r.d[6] = R(1); break;
                case F_C + 1: r.d[6] = R(-2); r.d[8] = R(2); break;
                case F_C + 2: r.d[6] = R(1); r.d[8] = R(-2); r.d[10] = R(1); break;
                case F_C + 3: r.d[7] = R(1); break;
                case F_C + 4: r.d[7] = R(-2); r.d[9] = R(2); break;
                case F_C + 5: r.d[7] = R(1); r.d[9] = R(-2); r.d[11] = R(1); break;
                default: break;
            }
        }
        return r;
    }
};

__device__ __forceinline__ double val_of(double x) { return x; }
__device__ __forceinline__ double val_of(float x) { return (double)x; }
template <typename R, int NT>
__device__ __forceinline__ double val_of(const Dn<R, NT>& x) {
    return (double)x.v;
}
// the real type under a dual (or the type itself)
template <typename N>
struct RealOf {
    using type = N;
};
template <typename R, int NT>
struct RealOf<Dn<R, NT>> {
    using type = R;
};

enum { GI_LOST = 0, GI_ON = 1, GI_DETECTED = 2, GI_OBSCURED = 3 };

// One interaction of the frozen path on the known surface S (N = double or float values, or
// DR<R> to carry derivatives): re-intersect, move the point, apply the surface's role.  At a refracting
// face refl_in = 0 refracts, 1 reflects, 2 decides with the trace's Fresnel draw (the forward
// pass), and *refl_out reports the choice.  Returns GI_LOST if the surface is not met any more,
// GI_DETECTED (q = local x, y) or GI_OBSCURED at the end of the path, GI_ON otherwise; *seg is
// the segment length and *front whether the ray met the front side.  The roughness tilt and the
// Fresnel decision use the trace's draws in the trace precision T.
template <typename T, typename N, typename SR>
__device__ __forceinline__ int g_interact(const Tables& tb, SR S, int4 si, double lam, uint4 wd, int refl_in,
                                          bool* refl_out, double eps, double ntol, V3<N>& p, V3<N>& d, N& qx, N& qy,
                                          double* seg, bool* front_out) {
    const int shape = si.x & 15, role = (si.x >> 4) & 15;
    const V3<N> pl = to_local_pt<N>(S, p), dl = to_local_vec<N>(S, d);
    LHit<N> h;
    bool ok = false, err = false;
    const N big = N(sizeof(typename RealOf<N>::type) == 4 ? 1.0e30 : 1.0e300);
    if (shape == SHAPE_SAG) {
        ok = hit_sag<false, true, N>(S, (si.x >> 8) & 15, (si.x >> 12) & 1, pl, dl, N(eps), big, N(ntol), h, err, nullptr);
        if (ok) {
            // one Newton step on the full sag: exact derivatives of the root in every parameter
            V3<N> x = pl + h.t * dl;
            N z, sl;
            if (sag_slope<N>(S, x.x * x.x + x.y * x.y, &z, &sl)) {
                const N fp = dl.z - sl * N(2) * (x.x * dl.x + x.y * dl.y);
                h.t = h.t - (x.z - z) / fp;
                x = pl + h.t * dl;
                if (sag_slope<N>(S, x.x * x.x + x.y * x.y, &z, &sl)) {
                    h.pl = x;
                    h.nl = unit(mk(N(-2) * x.x * sl, N(-2) * x.y * sl, N(1)));
                }
            }
        }
    } else if (shape == SHAPE_HEXCONE) {
        ok = hit_hexcone<N>(S, pl, dl, N(eps), big, h);
    }
    if (!ok || err) return GI_LOST;
    *seg = val_of(h.t);
    p = p + h.t * d;
    const V3<N> nw = unit(to_world_vec<N>(S, h.nl));
    const bool front = val_of(dot(d, nw)) < 0.0;
    *front_out = front;
    *refl_out = false;
    if (role == ROLE_FOCAL) {
        if (!front) return GI_OBSCURED;
        qx = h.pl.x;
        qy = h.pl.y;
        return GI_DETECTED;
    }
    if (role == ROLE_MIRROR) {
        if (!front) return GI_OBSCURED;
        const double* M = tb.mats + (size_t)si.y * MAT_REC;
        V3<N> nn = nw;
        const T sigma = (T)M[33];
        if (sigma > T(0)) {
            const T u1 = unit_open<T>(wd.y), u2 = unit_open<T>(wd.z);
            const T rad = t_sqrt(T(-2) * t_log(u1));
            T sn, cs;
            t_sincospi(T(2) * u2, &sn, &cs);
            const N g1 = N((double)(sigma * rad * cs)), g2 = N((double)(sigma * rad * sn));
            const N sgn = N(val_of(nw.z) >= 0.0 ? 1.0 : -1.0);
            const N aa = N(-1) / (sgn + nw.z);
            const N bb = nw.x * nw.y * aa;
            const V3<N> tt = mk(N(1) + sgn * nw.x * nw.x * aa, sgn * bb, N(0) - sgn * nw.x);
            const V3<N> bv = mk(bb, sgn + nw.y * nw.y * aa, N(0) - nw.y);
            nn = unit(nw + g1 * tt + g2 * bv);
        }
        d = unit(d - (N(2) * dot(d, nn)) * nn);
        return GI_ON;
    }
    // refracting face: the recorded choice, reflect or Snell
    const T na = refr_index<T>(tb.meds + (size_t)si.z * MED_REC, (T)lam);
    const T nb = refr_index<T>(tb.meds + (size_t)si.w * MED_REC, (T)lam);
    const T n1 = front ? na : nb, n2 = front ? nb : na;
    const V3<N> nf = front ? nw : N(-1) * nw;
    const N ci = N(0) - dot(d, nf);
    bool rv = refl_in == 1;
    if (refl_in == 2) rv = unit_open<T>(wd.x) < fresnel(n1, n2, (T)val_of(ci));
    *refl_out = rv;
    if (rv) {
        d = unit(d - (N(2) * dot(d, nf)) * nf);
    } else {
        const N eta = N((double)n1 / (double)n2);
        const N s2 = eta * eta * (N(1) - ci * ci);
        d = unit(eta * d + (eta * ci - t_sqrt(N(1) - s2)) * nf);
    }
    return GI_ON;
}

// Signed margin of the exit hexagon (apothem - max_k |x . u_k|) where the ray crosses the plane
// of the variant's exit surface; false if the ray does not head into it.
template <typename N, typename SR>
__device__ __forceinline__ bool g_exit_margin(SR S, V3<N> p, V3<N> d, N* m) {
    const V3<N> pl = to_local_pt<N>(S, p), dl = to_local_vec<N>(S, d);
    if (!(val_of(dl.z) < 0.0)) return false;
    const N t = N(0) - pl.z / dl.z;
    const V3<N> x = pl + t * dl;
    const N s60 = N(0.86602540378443864676);
    const N c0 = x.x, c1 = N(0.5) * x.x + s60 * x.y, c2 = N(-0.5) * x.x + s60 * x.y;
    N mx = t_abs(c0);
    if (val_of(t_abs(c1)) > val_of(mx)) mx = t_abs(c1);
    if (val_of(t_abs(c2)) > val_of(mx)) mx = t_abs(c2);
    *m = N(S[F_AP]) - mx;
    return true;
}

__device__ __forceinline__ bool g_differentiable(int4 si) {
    const int shape = si.x & 15, role = (si.x >> 4) & 15;
    return role == ROLE_MIRROR && (shape == SHAPE_SAG || shape == SHAPE_HEXCONE);
}

template <typename T>
__device__ __forceinline__ T sigmoid_t(T x) {
    return T(1) / (T(1) + (sizeof(T) == 4 ? (T)expf(-(float)x) : (T)exp(-(double)x)));
}

// Resident blocks of 128 threads per SM the register allocation must allow (FP32, FP64
// derivative passes).  FP32: 2 (255 registers; the 32-dish batch ran 162 ms per evaluation
// against 196 ms at 3 and 182 ms at 4, where the 16-slot duals spill more).
#ifndef ROBAST_GRAD_MIN_BLOCKS_F32
#define ROBAST_GRAD_MIN_BLOCKS_F32 2
#endif
#ifndef ROBAST_GRAD_MIN_BLOCKS_F64
#define ROBAST_GRAD_MIN_BLOCKS_F64 4
#endif
// T: the trace precision (nearest-hit search); R: the precision of the derivative passes.
template <typename T, typename R, int BLOCK, bool STAGED>
__global__ void __launch_bounds__(BLOCK, sizeof(R) == 4 ? ROBAST_GRAD_MIN_BLOCKS_F32 : ROBAST_GRAD_MIN_BLOCKS_F64)
    grad_kernel(GradArgs<T> A) {
    extern __shared__ __align__(16) unsigned char smem[];
    Tables tb = A.tab;
    if constexpr (STAGED) {
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
        tb.surf = stage(tb.surf, (size_t)tb.n_surf * REC * sizeof(T));
        tb.surf_i = reinterpret_cast<const int4*>(stage(tb.surf_i, (size_t)tb.n_surf * sizeof(int4)));
        tb.nodes = reinterpret_cast<const Node*>(stage(tb.nodes, (size_t)tb.n_nodes * sizeof(Node)));
        tb.prims = reinterpret_cast<const int*>(stage(tb.prims, (size_t)tb.n_prims * sizeof(int)));
        tb.variants = reinterpret_cast<const int4*>(stage(tb.variants, (size_t)tb.n_var * sizeof(int4)));
        tb.glob = reinterpret_cast<const int*>(stage(tb.glob, (size_t)tb.n_glob * sizeof(int)));
        tb.mats = reinterpret_cast<const double*>(stage(tb.mats, (size_t)tb.n_mat * MAT_REC * sizeof(double)));
        tb.meds = reinterpret_cast<const double*>(stage(tb.meds, (size_t)tb.n_med * MED_REC * sizeof(double)));
        __syncthreads();
    }
    const uint2 key = make_uint2((uint32_t)A.seed, (uint32_t)(A.seed >> 32));
    const long long n = A.n;
    const int nq = A.objective == 1 ? 1 : 2;  // objective terms per photon: (qx, qy) or the margin m
    int ids[GMAXB];
    float segs[GMAXB];  // segment length to each interaction (forward pass): where its derivative pass starts
    unsigned int u_fwd = 0, u_rep = 0, u_dual = 0;  // work units (when A.units is set)
    // photons of the current variant counted in a register, added when the variant changes
    int cnt_var = -1;
    unsigned long long cnt_n = 0ull;
    for (long long j = blockIdx.x * (long long)BLOCK + threadIdx.x; j < n; j += (long long)gridDim.x * BLOCK) {
        // in coherent order a warp's photons start close together and share their facets; every
        // photon keeps its index, random stream and contributions (integer sums: any order)
        const long long i = A.order ? (long long)A.order[j] : j;
        const V3<double> p0 = mk((double)A.o[i], (double)A.o[n + i], (double)A.o[2 * n + i]);
        const V3<double> d0 = mk((double)A.d[i], (double)A.d[n + i], (double)A.d[2 * n + i]);
        const T lam = A.lam[i];
        const int var = A.vop ? A.vop[i] : 0;
        const long long pid = A.first_id + i;
        if (var < 0 || var >= tb.n_var) continue;  // no variant to account it to
        unsigned long long* V = A.vals + (size_t)var * 16;
        // ---- 1. forward pass
        V3<double> p = p0, d = d0;
        double w = 1.0, qx = 0.0, qy = 0.0;
        unsigned long long refl = 0ull;  // refracting faces: bit k set = reflected at interaction k
        int K = 0, status = 0, first_diff = -1;
        bool untracked = false;
        for (int b = 0; status == 0; ++b) {
            Best<T> bst;
            bool overflow = false;
            nearest_hit<false>(tb, var, mk((T)p.x, (T)p.y, (T)p.z), mk((T)d.x, (T)d.y, (T)d.z), A.eps, A.newton_tol,
                               bst, overflow, nullptr);
            if (overflow || bst.err) {
                status = ST_ERROR;
                break;
            }
            if (bst.sid == 0x7fffffff) {
                status = ST_ESCAPED;
                break;
            }
            const int sid = bst.sid;
            const int4 si = tb.surf_i[sid];
            const int shape = si.x & 15, role = (si.x >> 4) & 15;
            if (role == ROLE_OBSC || shape == SHAPE_CYL || shape == SHAPE_BOX) {
                status = ST_OBSCURED;
                break;
            }
            if (K >= GMAXB) {  // longer than the path record: not differentiated
                untracked = true;
                status = ST_ERROR;
                break;
            }
            const uint4 wd = philox4x32_10(
                make_uint4((uint32_t)pid, (uint32_t)((unsigned long long)pid >> 32), (uint32_t)b, 0u), key);
            const double* S = A.surf64 + (size_t)sid * REC;
            double seg = 0.0;
            bool rev = false, front = true;
            const int gi = g_interact<T, double>(tb, S, si, (double)lam, wd, 2, &rev, (double)A.eps, A.newton_tol64, p,
                                                 d, qx, qy, &seg, &front);
            ++u_fwd;
            if (gi == GI_LOST) {
                status = ST_ERROR;  // the frozen path was lost
                break;
            }
            if (role == ROLE_REFRACT) {
                // bulk absorption of the segment through the medium the photon arrived in
                const T len = abs_length<T>(tb.meds + (size_t)(front ? si.z : si.w) * MED_REC, lam);
                if (len > T(0)) w *= exp(-seg / (double)len);
            }
            ids[K] = sid;
            segs[K] = (float)seg;
            if (rev) refl |= 1ull << K;
            if (first_diff < 0 && g_differentiable(si)) first_diff = K;
            ++K;
            if (gi == GI_DETECTED) {
                status = ST_DETECTED;
                break;
            }
            if (gi == GI_OBSCURED) {
                status = ST_OBSCURED;
                break;
            }
            if (role == ROLE_MIRROR) w *= refl_value(tb.mats + (size_t)si.y * MAT_REC, (double)lam);
            if (b + 1 >= A.max_bounces) status = ST_MAXB;
        }
        if (var != cnt_var) {
            if (cnt_var >= 0) fx_add_count(A.vals + (size_t)cnt_var * 16 + 2 * 7, cnt_n);
            cnt_var = var;
            cnt_n = 0ull;
        }
        ++cnt_n;
        if (untracked) fx_add(V + 2 * 6, 1.0);
        // ---- objective terms of this photon
        bool contributes = false;
        double coef = 0.0, m_val = 0.0;
        const int ex = tb.variants[var].w;
        if (A.objective != 1) {
            if (status == ST_DETECTED) {
                contributes = true;
                fx_add(V + 2 * 0, w);
                fx_add(V + 2 * 1, w * qx);
                fx_add(V + 2 * 2, w * qy);
                fx_add(V + 2 * 3, w * (qx * qx + qy * qy));
                fx_add(V + 2 * 5, 1.0);
            }
        } else if (status != ST_OBSCURED && status != ST_ERROR && status != ST_MAXB && ex >= 0) {
            double m;
            if (g_exit_margin<double>(A.surf64 + (size_t)ex * REC, p, d, &m)) {
                const double sg = 1.0 / (1.0 + exp(-m / A.tau));
                fx_add(V + 2 * 4, w * sg);
                coef = w * sg * (1.0 - sg) / A.tau;
                m_val = m;
                contributes = true;
            }
        }
        (void)m_val;
        if (!contributes || first_diff < 0) continue;
        // ---- 2. reverse sweep in precision R (the trace precision, or FP64 for paths through Bezier
        // cone walls): the replays and the dual-number interactions (the per-photon derivatives);
        // the sums over photons are fixed point
        using DN = DR<R>;
        R a[2][6];
        int k;  // the adjoint is with respect to the state before interaction k + 1 (after k)
        bool lost = false;
        const double ntol_r = sizeof(R) == 4 ? (double)A.newton_tol : A.newton_tol64;
        auto replay = [&](int upto, V3<R>& pr, V3<R>& dr) {
            // the state before interaction `upto`, from the photon's inputs
            pr = mk((R)A.o[i], (R)A.o[n + i], (R)A.o[2 * n + i]);
            dr = mk((R)A.d[i], (R)A.d[n + i], (R)A.d[2 * n + i]);
            u_rep += (unsigned)upto;
            for (int j = 0; j < upto; ++j) {
                const uint4 wd = philox4x32_10(
                    make_uint4((uint32_t)pid, (uint32_t)((unsigned long long)pid >> 32), (uint32_t)j, 0u), key);
                R qa, qb;
                double sg;
                bool rv, fr;
                // the trace's own table when R is its precision, else the FP64 records
                const R* Sj;
                if constexpr (sizeof(R) == sizeof(T))
                    Sj = reinterpret_cast<const R*>(tb.surf) + (size_t)ids[j] * REC;
                else
                    Sj = reinterpret_cast<const R*>(A.surf64) + (size_t)ids[j] * REC;
                if (g_interact<T, R>(tb, Sj, tb.surf_i[ids[j]], (double)lam, wd, (int)((refl >> j) & 1ull), &rv,
                                     (double)A.eps, ntol_r, pr, dr, qa, qb, &sg, &fr) == GI_LOST)
                    lost = true;
            }
        };
        // Dual state seeded on (position, direction).  The position is first moved along the ray
        // by t0, to just short of the hit, and expressed in world axes shifted to the origin of the
        // surface the pass evaluates (both in FP64), so the pass solves its hit from nearby in small
        // coordinates.  t0 is a constant: the derivative with respect to the direction before the
        // move is the one after it plus t0 times the position's (applied to the adjoint below).
        auto seed_state = [](V3<R> pv, V3<R> dv, const double* S, double t0, V3<DN>& ps, V3<DN>& ds) {
            ps = mk(DN((double)pv.x + t0 * (double)dv.x - S[F_O]), DN((double)pv.y + t0 * (double)dv.y - S[F_O + 1]),
                    DN((double)pv.z + t0 * (double)dv.z - S[F_O + 2]));
            ds = mk(DN(dv.x), DN(dv.y), DN(dv.z));
            ps.x.d[0] = R(1);
            ps.y.d[1] = R(1);
            ps.z.d[2] = R(1);
            ds.x.d[3] = R(1);
            ds.y.d[4] = R(1);
            ds.z.d[5] = R(1);
        };
        const double ntol_d = sizeof(R) == 4 ? (double)A.newton_tol : A.newton_tol64;
        // Where a derivative pass starts: short of the hit by more than the self-intersection
        // epsilon, the segment's FP32 record (6e-8 relative), the replay's rounding, and (an
        // asphere's Newton starts from its base quadric's first root ahead) 20 times the surface's
        // distance from that quadric (incidence cosines down to 0.05); never behind the state.
        auto start_of = [&](int j) {
            const double sg = (double)segs[j];
            const double dev = A.surf64[(size_t)ids[j] * REC + F_ADEV];
            return fmax(0.0, sg - (4.0 * (double)A.eps + (sizeof(R) == 4 ? 1e-5 : 1e-6) * sg + 20.0 * dev));
        };
        if (A.objective != 1) {
            // terminal adjoint: d(qx, qy) / d(state before the detecting interaction K - 1)
            V3<R> pr, dr;
            replay(K - 1, pr, dr);
            const double* S64 = A.surf64 + (size_t)ids[K - 1] * REC;
            const double t0 = start_of(K - 1);
            V3<DN> ps, ds;
            seed_state(pr, dr, S64, t0, ps, ds);
            const uint4 wd = philox4x32_10(
                make_uint4((uint32_t)pid, (uint32_t)((unsigned long long)pid >> 32), (uint32_t)(K - 1), 0u), key);
            DN qa(0.0), qb(0.0);
            double sg;
            bool rv, fr;
            const GRec<R> rec{S64, A.grec + (size_t)ids[K - 1] * 18, 0};
            if (g_interact<T, DN>(tb, rec, tb.surf_i[ids[K - 1]], (double)lam, wd, 0, &rv, (double)A.eps, ntol_d, ps,
                                  ds, qa, qb, &sg, &fr) == GI_LOST)
                lost = true;
            ++u_dual;
            for (int j = 0; j < 3; ++j) {
                a[0][j] = qa.d[j];
                a[1][j] = qb.d[j];
                a[0][3 + j] = qa.d[3 + j] + R(t0) * qa.d[j];
                a[1][3 + j] = qb.d[3 + j] + R(t0) * qb.d[j];
            }
            k = K - 2;
        } else {
            // terminal adjoint: d m / d(state after the last interaction)
            const double* Sx = A.surf64 + (size_t)ex * REC;
            V3<DN> ps, ds;
            seed_state(mk((R)p.x, (R)p.y, (R)p.z), mk((R)d.x, (R)d.y, (R)d.z), Sx, 0.0, ps, ds);
            DN m(0.0);
            g_exit_margin<DN>(GRec<R>{Sx, nullptr, 0}, ps, ds, &m);
            for (int j = 0; j < 6; ++j) {
                a[0][j] = m.d[j];
                a[1][j] = R(0);
            }
            k = K - 1;
        }
        // per-surface gradient of this photon's terms, flushed when the surface changes
        int cur = -1;
        R gs[2][10];
        auto flush = [&]() {
            if (cur < 0 || lost) return;
            const bool sag = (tb.surf_i[cur].x & 15) == SHAPE_SAG;
            const int base = sag ? 0 : 10, np = sag ? 10 : 6;
            unsigned long long* acc = A.acc + (size_t)cur * GRAD_SLOTS;
            for (int m = 0; m < np; ++m) {
                unsigned long long* c = acc + (size_t)(base + m) * 6;
                // contributions in the derivative precision (an FP32 one is converted with integer
                // operations); the weights and spot coordinates rounded to it
                if (A.objective != 1) {
                    const R wr = (R)w;
                    fx_add(c + 0, wr * ((R)qx * gs[0][m] + (R)qy * gs[1][m]));
                    fx_add(c + 2, wr * gs[0][m]);
                    fx_add(c + 4, wr * gs[1][m]);
                } else {
                    fx_add(c + 0, (R)coef * gs[0][m]);
                }
            }
        };
        for (; k >= first_diff && !lost; --k) {
            V3<R> pr, dr;
            replay(k, pr, dr);
            const int sid = ids[k];
            const int4 si = tb.surf_i[sid];
            const double* S64 = A.surf64 + (size_t)sid * REC;
            const double t0 = start_of(k);
            V3<DN> ps, ds;
            seed_state(pr, dr, S64, t0, ps, ds);
            const int mode = g_differentiable(si) ? ((si.x & 15) == SHAPE_SAG ? 1 : 2) : 0;
            const GRec<R> rec{S64, A.grec + (size_t)sid * 18, mode};
            const uint4 wd = philox4x32_10(
                make_uint4((uint32_t)pid, (uint32_t)((unsigned long long)pid >> 32), (uint32_t)k, 0u), key);
            DN qa(0.0), qb(0.0);
            double sg;
            bool rv, fr;
            if (g_interact<T, DN>(tb, rec, si, (double)lam, wd, (int)((refl >> k) & 1ull), &rv, (double)A.eps, ntol_d,
                                  ps, ds, qa, qb, &sg, &fr) == GI_LOST)
                lost = true;
            ++u_dual;
            const DN* out[6] = {&ps.x, &ps.y, &ps.z, &ds.x, &ds.y, &ds.z};
            if (mode) {
                if (sid != cur) {
                    flush();
                    cur = sid;
                    for (int c = 0; c < 2; ++c)
                        for (int m = 0; m < 10; ++m) gs[c][m] = R(0);
                }
                const int np = mode == 1 ? 10 : 6;
                for (int c = 0; c < nq; ++c)
                    for (int m = 0; m < np; ++m) {
                        R acc = R(0);
                        for (int j = 0; j < 6; ++j) acc += a[c][j] * out[j]->d[6 + m];
                        gs[c][m] += acc;
                    }
            }
            R na[2][6];
            for (int c = 0; c < nq; ++c)
                for (int j = 0; j < 6; ++j) {
                    R acc = R(0);
                    for (int i2 = 0; i2 < 6; ++i2) acc += a[c][i2] * out[i2]->d[j];
                    na[c][j] = acc;
                }
            for (int c = 0; c < nq; ++c)  // the move by t0: d/d(direction) += t0 d/d(position)
                for (int j = 0; j < 3; ++j) na[c][3 + j] += R(t0) * na[c][j];
            for (int c = 0; c < nq; ++c)
                for (int j = 0; j < 6; ++j) a[c][j] = na[c][j];
        }
        flush();
        // a derivative pass that no longer met its surface (a grazing hit the trace precision
        // resolves differently): the photon's remaining gradient is dropped and counted
        if (lost) fx_add(V + 2 * 6, 1.0);
    }
    if (cnt_var >= 0) fx_add_count(A.vals + (size_t)cnt_var * 16 + 2 * 7, cnt_n);
    if (A.units) {  // one atomic per warp and unit
        const unsigned fw = __reduce_add_sync(0xffffffffu, u_fwd), rp = __reduce_add_sync(0xffffffffu, u_rep),
                       du = __reduce_add_sync(0xffffffffu, u_dual);
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(A.units + 0, (unsigned long long)fw);
            atomicAdd(A.units + 1, (unsigned long long)rp);
            atomicAdd(A.units + 2, (unsigned long long)du);
        }
    }
}

// resident blocks of the gradient kernel per SM (0 if it cannot launch)
template <typename T, typename R>
static int grad_occupancy(size_t smem) {
    auto k = smem ? grad_kernel<T, R, 128, true> : grad_kernel<T, R, 128, false>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, 128, smem) != cudaSuccess) return 0;
    return nb;
}

template <typename T, typename R, int BLOCK, bool STAGED>
static cudaError_t launch_grad_one(const GradArgs<T>& a, int grid, size_t smem, cudaStream_t s) {
    auto k = grad_kernel<T, R, BLOCK, STAGED>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<grid, BLOCK, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace robast
