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
// Per photon the kernel re-traces the path (nearest hits in the trace's
// precision; per-bounce state recomputed, nothing stored) and re-intersects
// each surface it meets in FP64 forward-mode dual numbers carrying the
// derivatives with respect to the (at most 10) parameters of the one
// differentiable surface the path meets.  The duals are FP64 in both forms:
// derivatives of roots near tangency and the sums that combine them lose too
// much in FP32 (a few 1e-3 relative on the concentrator), and there is one
// dual intersection per bounce, so FP64 costs little here.  FP64 sums over photons give the value and the
// gradient in one pass (MSR: sum w q.dq and sum w dq, combined with qbar
// after the pass).
#include "dual.cuh"
#include "launch.h"

namespace robast {

constexpr int GNT = 10;

template <typename T>
using D = Dn<T, GNT>;
using DD = Dn<double, GNT>;

__device__ __forceinline__ V3<DD> lift(V3<double> a) { return mk(DD(a.x), DD(a.y), DD(a.z)); }
template <typename T>
__device__ __forceinline__ V3<T> value_of(const V3<DD>& a) {
    return mk((T)a.x.v, (T)a.y.v, (T)a.z.v);
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

// The dual-number record of surface sid: derivative slots only when it is the
// tracked surface (SAG mirror: tilt x, y, A1..A8; HEXCONE mirror: P0r, P0z,
// P1r, P1z, P2r, P2z).
template <typename T>
__device__ __forceinline__ void dual_record(const T* S, const T* G, int shape, bool tracked, D<T>* Sd) {
    for (int k = 0; k < REC; ++k) Sd[k] = D<T>(S[k]);
    if (!tracked) return;
    if (shape == SHAPE_SAG) {
        for (int j = 0; j < 9; ++j) {
            Sd[F_R + j].d[0] = G[j];
            Sd[F_R + j].d[1] = G[9 + j];
        }
        for (int i = 0; i < 8; ++i) Sd[F_A + i].d[2 + i] = T(1);
    } else {
        // power-basis coefficients of the Bezier profile in the control points
        Sd[F_C + 0].d[0] = T(1);
        Sd[F_C + 1].d[0] = T(-2);
        Sd[F_C + 1].d[2] = T(2);
        Sd[F_C + 2].d[0] = T(1);
        Sd[F_C + 2].d[2] = T(-2);
        Sd[F_C + 2].d[4] = T(1);
        Sd[F_C + 3].d[1] = T(1);
        Sd[F_C + 4].d[1] = T(-2);
        Sd[F_C + 4].d[3] = T(2);
        Sd[F_C + 5].d[1] = T(1);
        Sd[F_C + 5].d[3] = T(-2);
        Sd[F_C + 5].d[5] = T(1);
    }
}

template <typename T>
__device__ __forceinline__ T sigmoid_t(T x) {
    return T(1) / (T(1) + (sizeof(T) == 4 ? (T)expf(-(float)x) : (T)exp(-(double)x)));
}

// Resident blocks of 128 threads per SM the register allocation must allow.  The dual state
// spills at any cap; more warps hide the local-memory latency better.  Dish batch, 3.2e7
// photons (FP32 form): 1 (255 registers) 720 ms, 2 721, 3 973, 4 637, 5 640, 6 642, 8 658.
#ifndef ROBAST_GRAD_MIN_BLOCKS
#define ROBAST_GRAD_MIN_BLOCKS 4
#endif
template <typename T, int BLOCK, bool STAGED>
__global__ void __launch_bounds__(BLOCK, ROBAST_GRAD_MIN_BLOCKS) grad_kernel(GradArgs<T> A) {
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
    // per-variant sums held for the variant of this thread's current photons (photons of a
    // variant are contiguous, so a thread changes variant rarely): W, sum w qx, sum w qy,
    // sum w |q|^2, sum soft CE, n_det, untracked, n
    double vs[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int cur_var = -1;
    auto flush = [&]() {
        if (cur_var < 0) return;
        for (int k = 0; k < 8; ++k)
            if (vs[k] != 0.0) {
                atomicAdd(A.vals + (size_t)cur_var * 8 + k, vs[k]);
                vs[k] = 0.0;
            }
    };
    DD Sd[REC];
    for (long long i = blockIdx.x * (long long)BLOCK + threadIdx.x; i < n; i += (long long)gridDim.x * BLOCK) {
        V3<DD> p = lift(mk((double)A.o[i], (double)A.o[n + i], (double)A.o[2 * n + i]));
        V3<DD> d = lift(mk((double)A.d[i], (double)A.d[n + i], (double)A.d[2 * n + i]));
        const T lam = A.lam[i];
        const int var = A.vop ? A.vop[i] : 0;
        const long long pid = A.first_id + i;
        double w = 1.0;
        int tracked = -1, status = 0, extra = 0;
        DD qx(0), qy(0);
        if (var < 0 || var >= tb.n_var) continue;  // no variant to account it to
        if (var != cur_var) {
            flush();
            cur_var = var;
        }
        for (int b = 0; status == 0; ++b) {
            Best<T> bst;
            bool overflow = false;
            nearest_hit<false>(tb, var, value_of<T>(p), value_of<T>(d), A.eps, A.newton_tol, bst, overflow, nullptr);
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
            const bool diff = role == ROLE_MIRROR && (shape == SHAPE_SAG || shape == SHAPE_HEXCONE);
            if (diff && tracked < 0) tracked = sid;
            if (diff && sid != tracked) extra = 1;
            if (role == ROLE_OBSC || shape == SHAPE_CYL || shape == SHAPE_BOX) {
                status = ST_OBSCURED;
                break;
            }
            const double* S = A.surf64 + (size_t)sid * REC;
            dual_record<double>(S, A.grec + (size_t)sid * 18, shape, sid == tracked, Sd);
            const V3<DD> pl = to_local_pt<DD>(Sd, p), dl = to_local_vec<DD>(Sd, d);
            LHit<DD> h;
            bool ok = false, err = false;
            const DD big = DD(1.0e300);
            if (shape == SHAPE_SAG) {
                ok = hit_sag<false, DD>(Sd, (si.x >> 8) & 15, (si.x >> 12) & 1, pl, dl, DD((double)A.eps), big,
                                        DD(A.newton_tol64), h, err, nullptr);
                if (ok) {
                    // one Newton step on the full sag: exact derivatives of the root in every parameter
                    V3<DD> x = pl + h.t * dl;
                    DD z, sl;
                    if (sag_slope<DD>(Sd, x.x * x.x + x.y * x.y, &z, &sl)) {
                        const DD fp = dl.z - sl * DD(2) * (x.x * dl.x + x.y * dl.y);
                        h.t = h.t - (x.z - z) / fp;
                        x = pl + h.t * dl;
                        if (sag_slope<DD>(Sd, x.x * x.x + x.y * x.y, &z, &sl)) {
                            h.pl = x;
                            h.nl = unit(mk(DD(-2) * x.x * sl, DD(-2) * x.y * sl, DD(1)));
                        }
                    }
                }
            } else {
                ok = hit_hexcone<DD>(Sd, pl, dl, DD((double)A.eps), big, h);
            }
            if (!ok || err) {
                status = ST_ERROR;  // the frozen path was lost
                break;
            }
            p = p + h.t * d;
            const uint4 wd = philox4x32_10(
                make_uint4((uint32_t)pid, (uint32_t)((unsigned long long)pid >> 32), (uint32_t)b, 0u), key);
            const V3<DD> nw = unit(to_world_vec<DD>(Sd, h.nl));
            const bool front = dot(value_of<double>(d), value_of<double>(nw)) < 0.0;
            if (role == ROLE_FOCAL) {
                if (front) {
                    status = ST_DETECTED;
                    qx = h.pl.x;
                    qy = h.pl.y;
                } else {
                    status = ST_OBSCURED;
                }
                break;
            }
            if (role == ROLE_MIRROR) {
                if (!front) {
                    status = ST_OBSCURED;
                    break;
                }
                const double* M = tb.mats + (size_t)si.y * MAT_REC;
                w *= refl_value(M, (double)lam);
                V3<DD> nn = nw;
                const T sigma = (T)M[33];
                if (sigma > T(0)) {
                    // the trace's roughness draw, in its precision
                    const T u1 = unit_open<T>(wd.y), u2 = unit_open<T>(wd.z);
                    const T rad = t_sqrt(T(-2) * t_log(u1));
                    T sn, cs;
                    t_sincospi(T(2) * u2, &sn, &cs);
                    const DD g1 = DD((double)(sigma * rad * cs)), g2 = DD((double)(sigma * rad * sn));
                    const DD sgn = DD(nw.z.v >= 0.0 ? 1 : -1);
                    const DD aa = DD(-1) / (sgn + nw.z);
                    const DD bb = nw.x * nw.y * aa;
                    const V3<DD> tt = mk(DD(1) + sgn * nw.x * nw.x * aa, sgn * bb, -sgn * nw.x);
                    const V3<DD> bv = mk(bb, sgn + nw.y * nw.y * aa, -nw.y);
                    nn = unit(nw + g1 * tt + g2 * bv);
                }
                d = unit(d - (DD(2) * dot(d, nn)) * nn);
            } else {  // refracting face: bulk absorption weight, the trace's Fresnel decision, reflect or Snell
                const T len = abs_length<T>(tb.meds + (size_t)(front ? si.z : si.w) * MED_REC, lam);
                if (len > T(0)) w *= exp(-h.t.v / (double)len);
                const T na = refr_index<T>(tb.meds + (size_t)si.z * MED_REC, lam);
                const T nb = refr_index<T>(tb.meds + (size_t)si.w * MED_REC, lam);
                const T n1 = front ? na : nb, n2 = front ? nb : na;
                const V3<DD> nf = front ? nw : DD(-1) * nw;
                const DD ci = -dot(d, nf);
                if (unit_open<T>(wd.x) < fresnel(n1, n2, (T)ci.v)) {
                    d = unit(d - (DD(2) * dot(d, nf)) * nf);
                } else {
                    const DD eta = DD((double)n1 / (double)n2);
                    const DD s2 = eta * eta * (DD(1) - ci * ci);
                    d = unit(eta * d + (eta * ci - t_sqrt(DD(1) - s2)) * nf);
                }
            }
            if (b + 1 >= A.max_bounces) status = ST_MAXB;
        }
        vs[7] += 1.0;
        if (extra) vs[6] += 1.0;
        const int base = tracked >= 0 ? (((tb.surf_i[tracked].x & 15) == SHAPE_SAG) ? 0 : 10) : 0;
        const int nslot = tracked >= 0 ? (base == 0 ? 10 : 6) : 0;
        double* acc = A.acc + (size_t)tracked * 16 * 3;
        if (A.objective != 1) {
            if (status == ST_DETECTED) {
                const double x = (double)qx.v, y = (double)qy.v;
                vs[0] += w;
                vs[1] += w * x;
                vs[2] += w * y;
                vs[3] += w * (x * x + y * y);
                vs[5] += 1.0;
                for (int k = 0; k < nslot; ++k) {
                    const double gx = (double)qx.d[k], gy = (double)qy.d[k];
                    atomicAdd(acc + (base + k) * 3 + 0, w * (x * gx + y * gy));
                    atomicAdd(acc + (base + k) * 3 + 1, w * gx);
                    atomicAdd(acc + (base + k) * 3 + 2, w * gy);
                }
            }
        } else if (status != ST_OBSCURED && status != ST_ERROR && status != ST_MAXB) {
            const int ex = tb.variants[var].w;
            if (ex >= 0) {
                const double* S = A.surf64 + (size_t)ex * REC;
                dual_record<double>(S, A.grec + (size_t)ex * 18, SHAPE_SAG, false, Sd);
                const V3<DD> pl = to_local_pt<DD>(Sd, p), dl = to_local_vec<DD>(Sd, d);
                if (dl.z.v < T(0)) {
                    const DD t = -pl.z / dl.z;
                    const V3<DD> x = pl + t * dl;
                    const DD s60 = DD(0.86602540378443864676);
                    const DD c0 = x.x, c1 = DD(0.5) * x.x + s60 * x.y, c2 = DD(-0.5) * x.x + s60 * x.y;
                    DD mx = t_abs(c0);
                    if (t_abs(c1).v > mx.v) mx = t_abs(c1);
                    if (t_abs(c2).v > mx.v) mx = t_abs(c2);
                    const DD m = DD(S[F_AP]) - mx;
                    const double sg = 1.0 / (1.0 + exp(-m.v / A.tau));
                    vs[4] += w * sg;
                    const double coef = w * sg * (1.0 - sg) / A.tau;
                    for (int k = 0; k < nslot; ++k) atomicAdd(acc + (base + k) * 3, coef * (double)m.d[k]);
                }
            }
        }
    }
    flush();
}

// d_params[p] += d_obj * gradient, from the sums of the pass (the sums of the
// variant the parameter's surface belongs to)
__global__ void grad_finish(const double* acc, const double* vals_all, const int* surf_var, int n_params,
                            int objective, double d_obj, double* out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_params) return;
    const double* vals = vals_all + (size_t)surf_var[p / 16] * 8;
    const double W = vals[0];
    double g = 0.0;
    if (objective == 1) {
        g = vals[7] > 0 ? acc[3 * p] / vals[7] : 0.0;
    } else if (W > 0) {
        const double qx = vals[1] / W, qy = vals[2] / W;
        if (objective == 0) g = 2.0 / W * (acc[3 * p] - qx * acc[3 * p + 1] - qy * acc[3 * p + 2]);
        if (objective == 2) g = acc[3 * p + 1] / W;
        if (objective == 3) g = acc[3 * p + 2] / W;
    }
    out[p] += d_obj * g;
}

template <typename T, int BLOCK, bool STAGED>
static cudaError_t launch_grad_one(const GradArgs<T>& a, int grid, size_t smem, cudaStream_t s) {
    auto k = grad_kernel<T, BLOCK, STAGED>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<grid, BLOCK, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_grad_f32(const GradArgs<float>& a, int grid, size_t smem, cudaStream_t s) {
    return a.stage ? launch_grad_one<float, 128, true>(a, grid, smem, s) : launch_grad_one<float, 128, false>(a, grid, 0, s);
}
cudaError_t launch_grad_f64(const GradArgs<double>& a, int grid, size_t smem, cudaStream_t s) {
    return a.stage ? launch_grad_one<double, 128, true>(a, grid, smem, s)
                   : launch_grad_one<double, 128, false>(a, grid, 0, s);
}
cudaError_t launch_grad_finish(const double* acc, const double* vals, const int* surf_var, int n_params, int objective,
                               double d_obj, double* out, cudaStream_t s) {
    grad_finish<<<(n_params + 255) / 256, 256, 0, s>>>(acc, vals, surf_var, n_params, objective, d_obj, out);
    return cudaGetLastError();
}

}  // namespace robast
