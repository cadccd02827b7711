// Host side of the C ABI (include/robast.h): descriptor validation, the
// geometry compiler (tilted local frames, FP32/FP64 surface records,
// conservative bounding boxes, one BVH per variant), trace launches, the
// spot-diagram reduction and error reporting.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cooperative_groups.h>

#include "../../include/robast.h"
#include "launch.h"

using namespace robast;

// ------------------------------------------------------------------ errors
static thread_local std::string g_err;

static int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

static int cuda_fail(cudaError_t e, const char* what) {
    return fail(ROBAST_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CU(call, what)                                    \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

extern "C" const char* robast_last_error(void) { return g_err.c_str(); }
extern "C" const char* robast_version(void) { return "robast-gb300 0.1 (sm_103a)"; }

// --------------------------------------------------------------- geometry
struct robast_geom {
    int device = 0;
    int n_surf = 0, n_var = 0, n_mat = 0, n_med = 0;
    int n_nodes = 0, n_prims = 0, n_glob = 0;
    double length_scale = 1.0;
    void* dmem = nullptr;  // one allocation holding every table
    Tables tab32{}, tab64{};
    const double* grec64 = nullptr;    // per surface: d rows / d tilt_x, d rows / d tilt_y
    const int* surf_var = nullptr;    // variant of each surface
    std::vector<int> h_var, h_flags;  // host copies: variant, shape | role << 4 of each surface
    size_t smem32 = 0, smem64 = 0;  // bytes to stage each precision's tables
    int num_sms = 0;
    // per-launch work counters (a ring, so launches on several streams do not share one)
    unsigned long long* work = nullptr;
    std::atomic<unsigned> work_slot{0};
    // staging for robast_trace_host and scratch for reductions
    std::mutex mu;
    void* stage = nullptr;
    size_t stage_bytes = 0;
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    // stream-ordered scratch (the coherent-order sort) comes from this pool, which keeps its
    // memory between calls (the device's default pool would hand it back at every
    // synchronisation and re-map it on the next call)
    cudaMemPool_t pool = nullptr;
    cudaStream_t hstream[2] = {nullptr, nullptr};  // robast_trace_host's pipeline
    cudaEvent_t hevent = nullptr;
    void* pinned = nullptr;  // pinned host staging for the reductions' small copies
    size_t pinned_bytes = 0;
    // resident blocks per SM of each trace kernel with this geometry's staged tables, looked
    // up once: [precision 32/64][block 64/128/256/512][source mode]; 0 = not yet known
    std::atomic<int> bps_cache[2][4][2] = {};
    std::atomic<int> bps_retrace[2] = {};  // the FP64 re-trace kernel [source mode]
    unsigned feat = 0;  // the surface kinds and interactions the geometry uses (FT_* bits)
};

static const int kWorkSlots = 256;

namespace {

struct Box {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    void add(const double p[3]) {
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], p[k]);
            hi[k] = std::max(hi[k], p[k]);
        }
    }
    void add(const Box& b) {
        add(b.lo);
        add(b.hi);
    }
    double centre(int k) const { return 0.5 * (lo[k] + hi[k]); }
};

void mat3_mul(const double a[9], const double b[9], double c[9]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) c[3 * i + j] = a[3 * i] * b[j] + a[3 * i + 1] * b[3 + j] + a[3 * i + 2] * b[6 + j];
}

// Rows of the tilted frame: Ry(b)^T Rx(a)^T R (rotation about local x by a,
// then about the new local y by b).
void tilted_rows(const robast_surface_desc& s, double out[9]) {
    const double ca = std::cos(s.tilt[0]), sa = std::sin(s.tilt[0]);
    const double cb = std::cos(s.tilt[1]), sb = std::sin(s.tilt[1]);
    const double rxT[9] = {1, 0, 0, 0, ca, sa, 0, -sa, ca};
    const double ryT[9] = {cb, 0, -sb, 0, 1, 0, sb, 0, cb};
    double tmp[9];
    mat3_mul(rxT, s.rot, tmp);
    mat3_mul(ryT, tmp, out);
}

double aperture_bound(const robast_surface_desc& s) {
    switch (s.aperture) {
        case ROBAST_AP_CIRCLE: return s.ap[0];
        case ROBAST_AP_ANNULUS:
        case ROBAST_AP_SECTOR: return s.ap[1];
        case ROBAST_AP_HEXAGON: return s.ap[0] * 2.0 / std::sqrt(3.0);
        case ROBAST_AP_RECT: return std::sqrt(s.ap[0] * s.ap[0] + s.ap[1] * s.ap[1]);
    }
    return INFINITY;
}

bool any_asph(const robast_surface_desc& s) {
    for (int i = 0; i < 8; ++i)
        if (s.asph[i] != 0.0) return true;
    return false;
}

// Bound on the principal curvatures of a surface over the region its hits can lie in (the
// FP32 error estimate turns a hit-point error into a normal error with it): the largest of
// the meridional and sagittal curvatures of a sag surface sampled over 1.1x its aperture's
// bounding radius, 1 / radius for a cylinder, 0 for a box, the largest curvature of a cone's
// Bezier profile; times 1.1 for what the sampling (1024 points) misses.
double curvature_bound(const robast_surface_desc& s, double L) {
    const int NS = 1024;
    double kmax = 0.0;
    switch (s.shape) {
        case ROBAST_SHAPE_SAG: {
            const double c = s.curv, k1 = 1.0 + s.conic;
            double rmax = 1.1 * aperture_bound(s);
            if (k1 * c * c > 0.0) rmax = std::min(rmax, 0.999 / std::sqrt(k1 * c * c));
            if (!std::isfinite(rmax)) rmax = 10.0 * L;
            for (int k = 0; k <= NS; ++k) {
                const double r = rmax * k / NS, rho = r * r;
                const double arg = 1.0 - k1 * c * c * rho;
                if (arg <= 0.0) break;
                const double sq = std::sqrt(arg);
                double S = c / (2.0 * sq), dS = c * k1 * c * c / (4.0 * sq * sq * sq);
                double rp = 1.0;  // rho^(i-1)
                for (int i = 1; i <= 8; ++i) {
                    S += i * s.asph[i - 1] * rp;
                    if (i >= 2) dS += i * (i - 1) * s.asph[i - 1] * rp / rho;
                    rp *= rho;
                }
                if (rho == 0.0) dS = c * k1 * c * c / 4.0 + 2.0 * s.asph[1];
                const double z1 = 2.0 * r * S, z2 = 2.0 * S + 4.0 * rho * dS;  // dz/dr, d2z/dr2
                const double q = 1.0 + z1 * z1;
                const double km = std::fabs(z2) / (q * std::sqrt(q));
                const double ks = std::fabs(2.0 * S) / std::sqrt(q);  // (dz/dr) / (r sqrt q)
                kmax = std::max(kmax, std::max(km, ks));
            }
            break;
        }
        case ROBAST_SHAPE_CYLINDER: kmax = s.prm[0] > 0.0 ? 1.0 / s.prm[0] : 0.0; break;
        case ROBAST_SHAPE_BOX: kmax = 0.0; break;
        case ROBAST_SHAPE_HEXCONE: {
            const double ra1 = 2.0 * (s.prm[2] - s.prm[0]), ra2 = s.prm[0] - 2.0 * s.prm[2] + s.prm[4];
            const double za1 = 2.0 * (s.prm[3] - s.prm[1]), za2 = s.prm[1] - 2.0 * s.prm[3] + s.prm[5];
            for (int k = 0; k <= NS; ++k) {
                const double u = (double)k / NS;
                const double r1 = ra1 + 2.0 * ra2 * u, z1 = za1 + 2.0 * za2 * u;
                const double q = r1 * r1 + z1 * z1;
                if (q > 0.0) kmax = std::max(kmax, std::fabs(r1 * 2.0 * za2 - z1 * 2.0 * ra2) / (q * std::sqrt(q)));
            }
            break;
        }
    }
    return 1.1 * kmax;
}

double sag_eval(const robast_surface_desc& s, double rho, bool* ok) {
    const double arg = 1.0 - (1.0 + s.conic) * s.curv * s.curv * rho;
    if (arg < 0.0) {
        *ok = false;
        return 0.0;
    }
    double z = s.curv * rho / (1.0 + std::sqrt(arg)), rp = rho;
    for (int i = 0; i < 8; ++i) {
        z += s.asph[i] * rp;
        rp *= rho;
    }
    *ok = true;
    return z;
}

// local (x, y) bounding rectangle of a SAG aperture
void aperture_rect(const robast_surface_desc& s, double* x0, double* x1, double* y0, double* y1) {
    switch (s.aperture) {
        case ROBAST_AP_CIRCLE:
        case ROBAST_AP_ANNULUS: {
            const double r = aperture_bound(s);
            *x0 = *y0 = -r;
            *x1 = *y1 = r;
            return;
        }
        case ROBAST_AP_SECTOR: {
            // corners plus the axis extremes the arc passes through
            const double r0 = s.ap[0], r1 = s.ap[1], p0 = s.ap[2], p1 = s.ap[3];
            double xs[8], ys[8];
            int n = 0;
            for (double r : {r0, r1})
                for (double p : {p0, p1}) {
                    xs[n] = r * std::cos(p);
                    ys[n] = r * std::sin(p);
                    ++n;
                }
            *x0 = *x1 = xs[0];
            *y0 = *y1 = ys[0];
            for (int k = 1; k < n; ++k) {
                *x0 = std::min(*x0, xs[k]);
                *x1 = std::max(*x1, xs[k]);
                *y0 = std::min(*y0, ys[k]);
                *y1 = std::max(*y1, ys[k]);
            }
            for (int q = -4; q <= 8; ++q) {
                const double a = q * M_PI / 2.0;
                if (a >= p0 && a <= p1) {
                    *x0 = std::min(*x0, r1 * std::cos(a));
                    *x1 = std::max(*x1, r1 * std::cos(a));
                    *y0 = std::min(*y0, r1 * std::sin(a));
                    *y1 = std::max(*y1, r1 * std::sin(a));
                }
            }
            return;
        }
        case ROBAST_AP_HEXAGON:
            *x0 = -s.ap[0];
            *x1 = s.ap[0];
            *y0 = -s.ap[0] * 2.0 / std::sqrt(3.0);
            *y1 = -*y0;
            return;
        case ROBAST_AP_RECT:
            *x0 = -s.ap[0];
            *x1 = s.ap[0];
            *y0 = -s.ap[1];
            *y1 = s.ap[1];
            return;
    }
    *x0 = *y0 = -INFINITY;
    *x1 = *y1 = INFINITY;
}

// Local bounding box of a surface; false if unbounded (tested every bounce).
bool local_box(const robast_surface_desc& s, double lo[3], double hi[3]) {
    switch (s.shape) {
        case ROBAST_SHAPE_SAG: {
            if (s.aperture == ROBAST_AP_NONE) return false;
            aperture_rect(s, &lo[0], &hi[0], &lo[1], &hi[1]);
            // z range of the sag over the radii the aperture spans
            double rmin = 0.0;
            if (s.aperture == ROBAST_AP_ANNULUS || s.aperture == ROBAST_AP_SECTOR) rmin = s.ap[0];
            const double rmax = aperture_bound(s);
            double zlo = INFINITY, zhi = -INFINITY;
            const int N = 512;
            for (int k = 0; k <= N; ++k) {
                const double r = rmin + (rmax - rmin) * k / N;
                bool ok;
                const double z = sag_eval(s, r * r, &ok);
                if (!ok) continue;
                zlo = std::min(zlo, z);
                zhi = std::max(zhi, z);
            }
            if (!(zlo <= zhi)) zlo = zhi = 0.0;
            // sampling margin: a fraction of the range plus the step's slope bound
            const double m = 0.01 * (zhi - zlo) + 1e-9 * rmax;
            lo[2] = zlo - m;
            hi[2] = zhi + m;
            return true;
        }
        case ROBAST_SHAPE_CYLINDER:
            lo[0] = lo[1] = -s.prm[0];
            hi[0] = hi[1] = s.prm[0];
            lo[2] = 0.0;
            hi[2] = s.prm[1];
            return true;
        case ROBAST_SHAPE_BOX:
            for (int k = 0; k < 3; ++k) {
                lo[k] = -s.prm[k];
                hi[k] = s.prm[k];
            }
            return true;
        case ROBAST_SHAPE_HEXCONE: {
            const double rm = std::max({s.prm[0], s.prm[2], s.prm[4]}) * 2.0 / std::sqrt(3.0);
            lo[0] = lo[1] = -rm;
            hi[0] = hi[1] = rm;
            lo[2] = std::min({s.prm[1], s.prm[3], s.prm[5]});
            hi[2] = std::max({s.prm[1], s.prm[3], s.prm[5]});
            return true;
        }
    }
    return false;
}

// World box of the local box through the tilted frame, padded and rounded
// outwards to float.
Box world_box(const double rows[9], const double o[3], const double lo[3], const double hi[3], double pad) {
    Box b;
    for (int c = 0; c < 8; ++c) {
        const double l[3] = {(c & 1) ? hi[0] : lo[0], (c & 2) ? hi[1] : lo[1], (c & 4) ? hi[2] : lo[2]};
        double w[3];
        for (int k = 0; k < 3; ++k) w[k] = o[k] + rows[k] * l[0] + rows[3 + k] * l[1] + rows[6 + k] * l[2];
        b.add(w);
    }
    for (int k = 0; k < 3; ++k) {
        const double p = pad + 1e-6 * std::max(std::fabs(b.lo[k]), std::fabs(b.hi[k]));
        b.lo[k] = std::nextafter((double)(float)(b.lo[k] - p), -INFINITY);
        b.hi[k] = std::nextafter((double)(float)(b.hi[k] + p), INFINITY);
        b.lo[k] = (double)std::nextafterf((float)b.lo[k], -INFINITY);
        b.hi[k] = (double)std::nextafterf((float)b.hi[k], INFINITY);
    }
    return b;
}

// A BVH primitive: one surface and its box.  Every surface is one
// reference, masts included: splitting a slanted mast into segments with
// tighter boxes was measured on the dish workload and lost (2, 4, 6 and 16
// segments gave 11%, 15%, 13% and 22% more box tests per bounce than one and
// slower traces; the cylinder tests they save are fewer than the box tests
// the extra references add).
struct Ref {
    int sid;
    Box box;
};

double half_area(const Box& b) {
    const double dx = b.hi[0] - b.lo[0], dy = b.hi[1] - b.lo[1], dz = b.hi[2] - b.lo[2];
    return dx * dy + dy * dz + dz * dx;
}

// Binary build node: box, and either children a, a + 1 (b == 0) or a leaf
// with prims [a, a + b).
struct BuildNode {
    Box box;
    int a = 0, b = 0;
};

// Binned surface-area-heuristic build (16 bins per axis), leaves of <= 4.
struct BvhBuilder {
    const std::vector<Ref>& refs;
    std::vector<BuildNode>& nodes;
    std::vector<int>& prims;
    static const int kBins = 16, kMaxLeaf = 4;

    void set_box(int ni, const Box& b) { nodes[ni].box = b; }
    void make_leaf(int ni, const std::vector<int>& ids, int b, int e) {
        nodes[ni].a = (int)prims.size();
        nodes[ni].b = e - b;
        for (int k = b; k < e; ++k) prims.push_back(refs[ids[k]].sid);
    }
    // node ni covers ids[b, e) (indices into refs)
    void build(int ni, std::vector<int>& ids, int b, int e) {
        Box bb, cb;
        for (int k = b; k < e; ++k) {
            const Box& r = refs[ids[k]].box;
            bb.add(r);
            const double c[3] = {r.centre(0), r.centre(1), r.centre(2)};
            cb.add(c);
        }
        set_box(ni, bb);
        const int n = e - b;
        if (n <= 2) return make_leaf(ni, ids, b, e);
        double best = INFINITY;
        int bax = -1, bsplit = -1;
        for (int ax = 0; ax < 3; ++ax) {
            const double ext = cb.hi[ax] - cb.lo[ax];
            if (!(ext > 0.0)) continue;
            Box bin[kBins];
            int cnt[kBins] = {0};
            for (int k = b; k < e; ++k) {
                const Box& r = refs[ids[k]].box;
                int bi = (int)((r.centre(ax) - cb.lo[ax]) / ext * kBins);
                bi = std::min(kBins - 1, std::max(0, bi));
                bin[bi].add(r);
                ++cnt[bi];
            }
            Box lb[kBins];
            int lc[kBins];
            Box acc;
            int c = 0;
            for (int i = 0; i < kBins; ++i) {
                if (cnt[i]) acc.add(bin[i]);
                c += cnt[i];
                lb[i] = acc;
                lc[i] = c;
            }
            Box racc;
            int rc = 0;
            for (int i = kBins - 1; i > 0; --i) {
                if (cnt[i]) racc.add(bin[i]);
                rc += cnt[i];
                if (lc[i - 1] == 0 || rc == 0) continue;
                const double cost = half_area(lb[i - 1]) * lc[i - 1] + half_area(racc) * rc;
                if (cost < best) {
                    best = cost;
                    bax = ax;
                    bsplit = i;
                }
            }
        }
        if (bax < 0) {  // all centroids coincide: split in the middle of the list
            if (n <= kMaxLeaf) return make_leaf(ni, ids, b, e);
            bax = 0;
        }
        if (n <= kMaxLeaf && best >= half_area(bb) * n) return make_leaf(ni, ids, b, e);
        int mid;
        if (bsplit > 0) {
            const double ext = cb.hi[bax] - cb.lo[bax];
            auto it = std::partition(ids.begin() + b, ids.begin() + e, [&](int x) {
                int bi = (int)((refs[x].box.centre(bax) - cb.lo[bax]) / ext * kBins);
                bi = std::min(kBins - 1, std::max(0, bi));
                return bi < bsplit;
            });
            mid = (int)(it - ids.begin());
        } else {
            mid = b + n / 2;
        }
        if (mid == b || mid == e) mid = b + n / 2;
        const int left = (int)nodes.size();
        nodes.push_back(BuildNode{});
        nodes.push_back(BuildNode{});
        nodes[ni].a = left;
        nodes[ni].b = 0;
        build(left, ids, b, mid);
        build(left + 1, ids, mid, e);
    }
};

// Convert the binary build into the device layout (each node carries both
// children's boxes), preorder so that the root comes first.
void emit_nodes(const std::vector<BuildNode>& bn, std::vector<Node>& out) {
    auto child = [&](Node& nd, int k, int c, int ref_internal) {
        float* lo = k == 0 ? nd.lo0 : nd.lo1;
        float* hi = k == 0 ? nd.hi0 : nd.hi1;
        for (int j = 0; j < 3; ++j) {
            lo[j] = (float)bn[c].box.lo[j];
            hi[j] = (float)bn[c].box.hi[j];
        }
        int& ref = k == 0 ? nd.ref0 : nd.ref1;
        int& n = k == 0 ? nd.n0 : nd.n1;
        if (bn[c].b > 0) {
            ref = bn[c].a;
            n = bn[c].b;
        } else {
            ref = ref_internal;
            n = 0;
        }
    };
    const int base = (int)out.size();
    if (bn[0].b > 0) {  // a single leaf: wrap it, as both children (its surfaces are tested twice, harmlessly)
        Node nd{};
        child(nd, 0, 0, -1);
        child(nd, 1, 0, -1);
        out.push_back(nd);
        return;
    }
    // index map from build nodes (internal only) to output nodes
    std::vector<int> map(bn.size(), -1), order;
    std::vector<int> st{0};
    while (!st.empty()) {
        const int i = st.back();
        st.pop_back();
        map[i] = base + (int)order.size();
        order.push_back(i);
        for (int c : {bn[i].a + 1, bn[i].a})
            if (bn[c].b == 0) st.push_back(c);
    }
    out.resize(base + order.size());
    for (size_t k = 0; k < order.size(); ++k) {
        const int i = order[k];
        Node nd{};
        child(nd, 0, bn[i].a, map[bn[i].a]);
        child(nd, 1, bn[i].a + 1, map[bn[i].a + 1]);
        out[base + k] = nd;
    }
}

int validate(const robast_geom_desc* d) {
    if (!d) return fail(ROBAST_E_NULL, "robast_build_geometry: desc is NULL");
    if (d->n_surfaces <= 0 || !d->surfaces)
        return fail(ROBAST_E_INVALID, "robast_build_geometry: need n_surfaces > 0 and a surface array");
    if (d->n_materials < 0 || d->n_media < 0 || (d->n_materials > 0 && !d->materials) ||
        (d->n_media > 0 && !d->media))
        return fail(ROBAST_E_INVALID, "robast_build_geometry: material/medium counts and arrays disagree");
    if (!(d->length_scale > 0.0) || !std::isfinite(d->length_scale))
        return fail(ROBAST_E_INVALID, "robast_build_geometry: length_scale must be finite and > 0");
    const int nv = d->variant_offsets ? d->n_variants : 1;
    if (d->variant_offsets) {
        if (d->n_variants <= 0) return fail(ROBAST_E_INVALID, "robast_build_geometry: n_variants must be > 0");
        if (d->variant_offsets[0] != 0 || d->variant_offsets[nv] != d->n_surfaces)
            return fail(ROBAST_E_INVALID, "robast_build_geometry: variant_offsets must run from 0 to n_surfaces");
        for (int v = 0; v < nv; ++v)
            if (d->variant_offsets[v + 1] < d->variant_offsets[v])
                return fail(ROBAST_E_INVALID, "robast_build_geometry: variant_offsets must be non-decreasing");
    }
    for (int i = 0; i < d->n_materials; ++i) {
        const robast_material_desc& m = d->materials[i];
        if (m.n < 1 || m.n > ROBAST_MAX_TABLE)
            return fail(ROBAST_E_INVALID, "material %d: table size %d outside 1..%d", i, m.n, ROBAST_MAX_TABLE);
        for (int k = 0; k + 1 < m.n; ++k)
            if (!(m.lam[k + 1] > m.lam[k]))
                return fail(ROBAST_E_INVALID, "material %d: wavelengths must increase", i);
        if (!(m.sigma >= 0.0)) return fail(ROBAST_E_INVALID, "material %d: sigma must be >= 0", i);
    }
    for (int i = 0; i < d->n_media; ++i) {
        const robast_medium_desc& m = d->media[i];
        if (m.n_abs < 0 || m.n_abs > ROBAST_MAX_TABLE)
            return fail(ROBAST_E_INVALID, "medium %d: absorption table size %d outside 0..%d", i, m.n_abs, ROBAST_MAX_TABLE);
        for (int k = 0; k < m.n_abs; ++k) {
            if (!(m.abs_len[k] > 0.0)) return fail(ROBAST_E_INVALID, "medium %d: absorption lengths must be > 0", i);
            if (k + 1 < m.n_abs && !(m.abs_lam[k + 1] > m.abs_lam[k]))
                return fail(ROBAST_E_INVALID, "medium %d: absorption wavelengths must increase", i);
        }
    }
    for (int i = 0; i < d->n_surfaces; ++i) {
        const robast_surface_desc& s = d->surfaces[i];
        if (s.shape < 0 || s.shape > 3) return fail(ROBAST_E_INVALID, "surface %d: unknown shape %d", i, s.shape);
        if (s.role < 0 || s.role > 3) return fail(ROBAST_E_INVALID, "surface %d: unknown role %d", i, s.role);
        if (s.aperture < 0 || s.aperture > 5)
            return fail(ROBAST_E_INVALID, "surface %d: unknown aperture %d", i, s.aperture);
        if (s.role == ROBAST_ROLE_MIRROR && (s.material < 0 || s.material >= d->n_materials))
            return fail(ROBAST_E_INVALID, "surface %d: material %d out of range", i, s.material);
        if (s.role == ROBAST_ROLE_REFRACT && (s.medium_front < 0 || s.medium_front >= d->n_media ||
                                              s.medium_back < 0 || s.medium_back >= d->n_media))
            return fail(ROBAST_E_INVALID, "surface %d: medium index out of range", i);
        // orthonormal frame
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                const double dp = s.rot[3 * r] * s.rot[3 * c] + s.rot[3 * r + 1] * s.rot[3 * c + 1] +
                                  s.rot[3 * r + 2] * s.rot[3 * c + 2];
                if (std::fabs(dp - (r == c ? 1.0 : 0.0)) > 1e-9)
                    return fail(ROBAST_E_INVALID, "surface %d: rot is not orthonormal", i);
            }
        if (s.shape == ROBAST_SHAPE_SAG) {
            if (s.aperture == ROBAST_AP_SECTOR && !(s.ap[3] > s.ap[2] && s.ap[3] - s.ap[2] <= M_PI + 1e-12))
                return fail(ROBAST_E_INVALID, "surface %d: sector needs phi0 < phi1 <= phi0 + pi", i);
            if ((s.aperture == ROBAST_AP_ANNULUS || s.aperture == ROBAST_AP_SECTOR) && !(s.ap[1] > s.ap[0] && s.ap[0] >= 0))
                return fail(ROBAST_E_INVALID, "surface %d: need 0 <= r_min < r_max", i);
            if ((s.aperture == ROBAST_AP_CIRCLE || s.aperture == ROBAST_AP_HEXAGON) && !(s.ap[0] > 0))
                return fail(ROBAST_E_INVALID, "surface %d: aperture size must be > 0", i);
            if (s.aperture == ROBAST_AP_RECT && !(s.ap[0] > 0 && s.ap[1] > 0))
                return fail(ROBAST_E_INVALID, "surface %d: rectangle half widths must be > 0", i);
            if (any_asph(s) && s.aperture == ROBAST_AP_NONE)
                return fail(ROBAST_E_INVALID, "surface %d: an aspheric surface needs a bounded aperture", i);
        } else if (s.shape == ROBAST_SHAPE_CYLINDER) {
            if (!(s.prm[0] > 0 && s.prm[1] > 0))
                return fail(ROBAST_E_INVALID, "surface %d: cylinder radius and length must be > 0", i);
        } else if (s.shape == ROBAST_SHAPE_BOX) {
            if (!(s.prm[0] > 0 && s.prm[1] > 0 && s.prm[2] > 0))
                return fail(ROBAST_E_INVALID, "surface %d: box half extents must be > 0", i);
        } else {
            if (!(s.prm[0] > 0 && s.prm[4] > 0 && s.prm[5] != s.prm[1]))
                return fail(ROBAST_E_INVALID, "surface %d: Bezier cone needs positive radii and height", i);
        }
    }
    return 0;
}

}  // namespace

static size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

extern "C" int robast_build_geometry(const robast_geom_desc* d, robast_geom** out) {
    if (!out) return fail(ROBAST_E_NULL, "robast_build_geometry: out is NULL");
    *out = nullptr;
    int rc = validate(d);
    if (rc) return rc;
    const int ns = d->n_surfaces;
    const int nv = d->variant_offsets ? d->n_variants : 1;
    const double L = d->length_scale;

    std::vector<double> rec64((size_t)ns * REC, 0.0);
    std::vector<float> rec32((size_t)ns * REC, 0.0f);
    std::vector<int4> reci(ns);
    std::vector<std::vector<Ref>> refs_of(ns);  // BVH references per surface; empty = unbounded
    std::vector<double> grec64((size_t)ns * 18, 0.0);
    unsigned feat = 0;
    for (int i = 0; i < ns; ++i) {
        const robast_surface_desc& s = d->surfaces[i];
        double* R = &rec64[(size_t)i * REC];
        double rows[9];
        tilted_rows(s, rows);
        for (int k = 0; k < 3; ++k) R[F_O + k] = s.origin[k];
        for (int k = 0; k < 9; ++k) R[F_R + k] = rows[k];
        const bool asph = s.shape == ROBAST_SHAPE_SAG && any_asph(s);
        switch (s.shape) {
            case ROBAST_SHAPE_SAG: {
                R[F_C] = s.curv;
                R[F_K1] = 1.0 + s.conic;
                for (int k = 0; k < 8; ++k) R[F_A + k] = s.asph[k];
                const double rb = 1.1 * aperture_bound(s);
                R[F_RB2] = rb * rb;
                double dev = 0.0, r2k = 1.0;
                for (int k = 0; k < 8; ++k) {
                    r2k *= rb * rb;
                    if (s.asph[k] != 0.0) dev += std::fabs(s.asph[k]) * r2k;  // no 0 x inf for unbounded
                }
                R[F_ADEV] = dev;
                double* A = R + F_AP;
                R[F_APR] = (s.aperture == ROBAST_AP_ANNULUS || s.aperture == ROBAST_AP_SECTOR) ? s.ap[0] : 0.0;
                R[F_APR + 1] = s.aperture == ROBAST_AP_CIRCLE ? s.ap[0]
                               : (s.aperture == ROBAST_AP_ANNULUS || s.aperture == ROBAST_AP_SECTOR) ? s.ap[1]
                                                                                                      : 0.0;
                switch (s.aperture) {
                    case ROBAST_AP_CIRCLE: A[0] = s.ap[0] * s.ap[0]; break;
                    case ROBAST_AP_ANNULUS:
                        A[0] = s.ap[0] * s.ap[0];
                        A[1] = s.ap[1] * s.ap[1];
                        break;
                    case ROBAST_AP_SECTOR:
                        A[0] = s.ap[0] * s.ap[0];
                        A[1] = s.ap[1] * s.ap[1];
                        A[2] = std::cos(s.ap[2]);
                        A[3] = std::sin(s.ap[2]);
                        A[4] = std::cos(s.ap[3]);
                        A[5] = std::sin(s.ap[3]);
                        break;
                    case ROBAST_AP_HEXAGON: A[0] = s.ap[0]; break;
                    case ROBAST_AP_RECT:
                        A[0] = s.ap[0];
                        A[1] = s.ap[1];
                        break;
                }
                break;
            }
            case ROBAST_SHAPE_CYLINDER:
                R[F_C] = s.prm[0];
                R[F_K1] = s.prm[1];
                break;
            case ROBAST_SHAPE_BOX:
                for (int k = 0; k < 3; ++k) R[F_C + k] = s.prm[k];
                break;
            case ROBAST_SHAPE_HEXCONE: {
                const double r0 = s.prm[0], z0 = s.prm[1], r1 = s.prm[2], z1 = s.prm[3], r2 = s.prm[4], z2 = s.prm[5];
                R[F_C + 0] = r0;
                R[F_C + 1] = 2.0 * (r1 - r0);
                R[F_C + 2] = r0 - 2.0 * r1 + r2;
                R[F_C + 3] = z0;
                R[F_C + 4] = 2.0 * (z1 - z0);
                R[F_C + 5] = z0 - 2.0 * z1 + z2;
                break;
            }
        }
        R[F_KAP] = curvature_bound(s, L);
        for (int k = 0; k < REC; ++k) rec32[(size_t)i * REC + k] = (float)R[k];
        // the FP32 origin as a pair: its rounding error in the low slots
        for (int k = 0; k < 3; ++k) rec32[(size_t)i * REC + F_OL + k] = (float)(s.origin[k] - (double)(float)s.origin[k]);
        {
            // derivatives of the tilted rows Ry(b)^T Rx(a)^T R with respect to a and b
            const double ca = std::cos(s.tilt[0]), sa = std::sin(s.tilt[0]);
            const double cb = std::cos(s.tilt[1]), sb = std::sin(s.tilt[1]);
            const double rxT[9] = {1, 0, 0, 0, ca, sa, 0, -sa, ca}, drxT[9] = {0, 0, 0, 0, -sa, ca, 0, -ca, -sa};
            const double ryT[9] = {cb, 0, -sb, 0, 1, 0, sb, 0, cb}, dryT[9] = {-sb, 0, -cb, 0, 0, 0, cb, 0, -sb};
            double t1[9], t2[9];
            mat3_mul(drxT, s.rot, t1);
            mat3_mul(ryT, t1, t2);  // d/da
            for (int k = 0; k < 9; ++k) grec64[(size_t)i * 18 + k] = t2[k];
            mat3_mul(rxT, s.rot, t1);
            mat3_mul(dryT, t1, t2);  // d/db
            for (int k = 0; k < 9; ++k) grec64[(size_t)i * 18 + 9 + k] = t2[k];
        }
        // a plane whose tilted frame has only 0 and +-1 entries: its world normal comes out exact in
        // FP32 (the FP32 error estimate then adds no rounding of the normal)
        bool exact_n = s.shape == ROBAST_SHAPE_SAG && s.curv == 0.0 && !asph;
        for (int k = 0; k < 9 && exact_n; ++k) exact_n = rows[k] == 0.0 || rows[k] == 1.0 || rows[k] == -1.0;
        reci[i] = make_int4(s.shape | (s.role << 4) | (s.aperture << 8) | ((asph ? 1 : 0) << 12) |
                                ((exact_n ? 1 : 0) << 13),
                            s.material, s.medium_front, s.medium_back);
        feat |= (asph ? (unsigned)FT_ASPH : 0u) | (s.shape == ROBAST_SHAPE_CYLINDER ? (unsigned)FT_CYL : 0u) |
                (s.shape == ROBAST_SHAPE_BOX ? (unsigned)FT_BOX : 0u) |
                (s.shape == ROBAST_SHAPE_HEXCONE ? (unsigned)FT_CONE : 0u) |
                (s.role == ROBAST_ROLE_REFRACT ? (unsigned)FT_REFR : 0u);
        double lo[3], hi[3];
        if (local_box(s, lo, hi)) refs_of[i].push_back(Ref{i, world_box(rows, s.origin, lo, hi, 1e-6 * L)});
    }
    // BVH per variant; unbounded surfaces go to a per-variant list
    std::vector<Node> nodes;
    std::vector<int> prims, glob;
    std::vector<int4> vars(nv);
    for (int v = 0; v < nv; ++v) {
        const int s0 = d->variant_offsets ? d->variant_offsets[v] : 0;
        const int s1 = d->variant_offsets ? d->variant_offsets[v + 1] : ns;
        std::vector<Ref> refs;
        const int g0 = (int)glob.size();
        for (int s = s0; s < s1; ++s) {
            if (refs_of[s].empty())
                glob.push_back(s);
            else
                refs.insert(refs.end(), refs_of[s].begin(), refs_of[s].end());
        }
        int root = -1;
        if (!refs.empty()) {
            std::vector<int> ids(refs.size());
            for (size_t k = 0; k < ids.size(); ++k) ids[k] = (int)k;
            std::vector<BuildNode> bn(1);
            BvhBuilder bb{refs, bn, prims};
            bb.build(0, ids, 0, (int)ids.size());
            root = (int)nodes.size();
            emit_nodes(bn, nodes);
        }
        // .w: the variant's exit surface (first focal plane with a hexagonal aperture), for soft CE
        int exit_sid = -1;
        for (int s = s0; s < s1 && exit_sid < 0; ++s) {
            const robast_surface_desc& q = d->surfaces[s];
            if (q.role == ROBAST_ROLE_FOCAL && q.shape == ROBAST_SHAPE_SAG && q.aperture == ROBAST_AP_HEXAGON &&
                q.curv == 0.0 && !any_asph(q))
                exit_sid = s;
        }
        vars[v] = make_int4(root, g0, (int)glob.size() - g0, exit_sid);
    }
    std::vector<double> mats((size_t)std::max(1, d->n_materials) * MAT_REC, 0.0);
    for (int i = 0; i < d->n_materials; ++i) {
        const robast_material_desc& m = d->materials[i];
        double* M = &mats[(size_t)i * MAT_REC];
        M[0] = m.n;
        for (int k = 0; k < m.n; ++k) {
            M[1 + k] = m.lam[k];
            M[17 + k] = m.refl[k];
        }
        M[33] = m.sigma;
    }
    std::vector<float> mats32(mats.size());
    for (size_t k = 0; k < mats.size(); ++k) mats32[k] = (float)mats[k];
    std::vector<double> meds((size_t)std::max(1, d->n_media) * MED_REC, 0.0);
    for (int i = 0; i < d->n_media; ++i) {
        double* M = &meds[(size_t)i * MED_REC];
        M[0] = d->media[i].n_const;
        for (int k = 0; k < 3; ++k) {
            M[1 + k] = d->media[i].B[k];
            M[4 + k] = d->media[i].C[k];
        }
        M[7] = d->media[i].n_abs;
        for (int k = 0; k < d->media[i].n_abs; ++k) {
            M[8 + k] = d->media[i].abs_lam[k];
            M[24 + k] = d->media[i].abs_len[k];
        }
    }
    if (glob.empty()) glob.push_back(0);
    if (prims.empty()) prims.push_back(0);
    if (nodes.empty()) nodes.push_back(Node{});

    // one device allocation: [rec64 | rec32 | reci | nodes | prims | vars | glob | mats | meds | mats32 | work | ...]
    const size_t b64 = align16(rec64.size() * 8), b32 = align16(rec32.size() * 4), bi = align16(reci.size() * 16);
    const size_t bn = align16(nodes.size() * sizeof(Node)), bp = align16(prims.size() * 4);
    const size_t bv = align16(vars.size() * 16), bg = align16(glob.size() * 4);
    std::vector<float> meds32(meds.size());
    for (size_t k = 0; k < meds.size(); ++k) meds32[k] = (float)meds[k];
    const size_t bm = align16(mats.size() * 8), bd = align16(meds.size() * 8), bm32 = align16(mats32.size() * 4);
    const size_t bd32 = align16(meds32.size() * 4);
    const size_t bw = kWorkSlots * 8;
    const size_t bg64 = align16(grec64.size() * 8);
    std::vector<int> surf_var(ns, 0);
    for (int v = 0; v < nv; ++v) {
        const int s0 = d->variant_offsets ? d->variant_offsets[v] : 0;
        const int s1 = d->variant_offsets ? d->variant_offsets[v + 1] : ns;
        for (int s = s0; s < s1; ++s) surf_var[s] = v;
    }
    const size_t bsv = align16(surf_var.size() * 4);
    const size_t total = b64 + b32 + bi + bn + bp + bv + bg + bm + bd + bm32 + bd32 + bw + bg64 + bsv;

    robast_geom* g = new (std::nothrow) robast_geom();
    if (!g) return fail(ROBAST_E_OOM, "robast_build_geometry: host allocation failed");
    cudaError_t e = cudaGetDevice(&g->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    if (e == cudaSuccess) e = cudaMalloc(&g->dmem, total);
    if (e == cudaSuccess) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = g->device;
        e = cudaMemPoolCreate(&g->pool, &props);
        if (e == cudaSuccess) {
            unsigned long long keep = ~0ull;  // keep whatever was used until the geometry is freed
            e = cudaMemPoolSetAttribute(g->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        if (e != cudaSuccess) {
            if (g->pool) cudaMemPoolDestroy(g->pool);
            g->pool = nullptr;
            cudaFree(g->dmem);
            g->dmem = nullptr;
        }
    }
    if (e != cudaSuccess) {
        delete g;
        return e == cudaErrorMemoryAllocation ? fail(ROBAST_E_OOM, "robast_build_geometry: cudaMalloc of %zu bytes failed", total)
                                              : cuda_fail(e, "robast_build_geometry");
    }
    std::vector<unsigned char> host(total, 0);
    size_t off = 0;
    auto put = [&](const void* src, size_t bytes, size_t padded) {
        std::memcpy(host.data() + off, src, bytes);
        const size_t at = off;
        off += padded;
        return at;
    };
    const size_t o64 = put(rec64.data(), rec64.size() * 8, b64);
    const size_t o32 = put(rec32.data(), rec32.size() * 4, b32);
    const size_t oi = put(reci.data(), reci.size() * 16, bi);
    const size_t on = put(nodes.data(), nodes.size() * sizeof(Node), bn);
    const size_t op = put(prims.data(), prims.size() * 4, bp);
    const size_t ov = put(vars.data(), vars.size() * 16, bv);
    const size_t og = put(glob.data(), glob.size() * 4, bg);
    const size_t om = put(mats.data(), mats.size() * 8, bm);
    const size_t od = put(meds.data(), meds.size() * 8, bd);
    const size_t om32 = put(mats32.data(), mats32.size() * 4, bm32);
    put(meds32.data(), meds32.size() * 4, bd32);  // right after the FP32 material records (meds32 in trace.cuh)
    const size_t ow = off;
    off += bw;
    const size_t og64 = put(grec64.data(), grec64.size() * 8, bg64);
    const size_t osv = put(surf_var.data(), surf_var.size() * 4, bsv);
    e = cudaMemcpy(g->dmem, host.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(g->dmem);
        cudaMemPoolDestroy(g->pool);
        delete g;
        return cuda_fail(e, "robast_build_geometry: upload");
    }
    unsigned char* base = static_cast<unsigned char*>(g->dmem);
    Tables t{};
    t.surf_i = reinterpret_cast<const int4*>(base + oi);
    t.nodes = reinterpret_cast<const Node*>(base + on);
    t.prims = reinterpret_cast<const int*>(base + op);
    t.variants = reinterpret_cast<const int4*>(base + ov);
    t.glob = reinterpret_cast<const int*>(base + og);
    t.mats = reinterpret_cast<const double*>(base + om);
    t.meds = reinterpret_cast<const double*>(base + od);
    t.mats32 = reinterpret_cast<const float*>(base + om32);
    t.n_surf = ns;
    t.n_nodes = (int)nodes.size();
    t.n_prims = (int)prims.size();
    t.n_var = nv;
    t.n_glob = (int)glob.size();
    t.n_mat = std::max(1, d->n_materials);
    t.n_med = std::max(1, d->n_media);
    g->tab64 = t;
    g->tab64.surf = base + o64;
    g->tab64.surf32 = reinterpret_cast<const float*>(base + o32);  // the FP64 search's FP32 screens
    g->tab32 = t;
    g->tab32.surf = base + o32;
    g->work = reinterpret_cast<unsigned long long*>(base + ow);
    g->grec64 = reinterpret_cast<const double*>(base + og64);
    g->surf_var = reinterpret_cast<const int*>(base + osv);
    g->smem64 = b64 + bi + bn + bp + bv + bg + bm + bd;
    g->smem32 = b32 + bi + bn + bp + bv + bg + bm + bd + bm32 + bd32;
    g->n_surf = ns;
    g->n_var = nv;
    g->h_var = surf_var;
    g->h_flags.resize(ns);
    for (int i = 0; i < ns; ++i) g->h_flags[i] = d->surfaces[i].shape | (d->surfaces[i].role << 4);
    g->n_mat = d->n_materials;
    g->n_med = d->n_media;
    g->n_nodes = (int)nodes.size();
    g->n_prims = (int)prims.size();
    g->n_glob = (int)glob.size();
    g->length_scale = L;
    g->feat = feat;
    *out = g;
    return 0;
}

extern "C" void robast_free_geometry(robast_geom* g) {
    if (!g) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(g->device);
    cudaDeviceSynchronize();
    cudaFree(g->dmem);
    if (g->stage) cudaFree(g->stage);
    if (g->scratch) cudaFree(g->scratch);
    if (g->pinned) cudaFreeHost(g->pinned);
    if (g->pool) cudaMemPoolDestroy(g->pool);
    for (int k = 0; k < 2; ++k)
        if (g->hstream[k]) cudaStreamDestroy(g->hstream[k]);
    if (g->hevent) cudaEventDestroy(g->hevent);
    cudaSetDevice(prev);
    delete g;
}

extern "C" int robast_geometry_info(const robast_geom* g, int32_t* n_surfaces, int32_t* n_variants,
                                    int32_t* n_bvh_nodes) {
    if (!g) return fail(ROBAST_E_NULL, "robast_geometry_info: g is NULL");
    if (n_surfaces) *n_surfaces = g->n_surf;
    if (n_variants) *n_variants = g->n_var;
    if (n_bvh_nodes) *n_bvh_nodes = g->n_nodes;
    return 0;
}

// ------------------------------------------------------------------ trace
extern "C" void robast_trace_opts_default(robast_trace_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->precision = 32;
    o->max_bounces = 100;
}

// Shared memory one block may use for staged tables.
static const size_t kSmemCap = 200 * 1024;

struct robast_sources {
    int device = 0;
    int n_groups = 0;
    long long n_photons = 0;
    SrcGroup* d_groups = nullptr;
    // the accuracy guard's re-trace queue: [4] u64 header (entries appended, spare), then
    // qcap photon indices
    unsigned long long* d_queue = nullptr;
    long long qcap = 0;
    // the coherent order of a chunk of qcap photons: their generated origins (x, y in FP32) and
    // the counting sort's scratch (order_scratch_bytes(qcap))
    float* d_xy = nullptr;
    void* d_ord = nullptr;
};

// The accuracy guard re-traces a photon whose error estimate exceeds this fraction of a bound.
// Measured with the guard off on 2.5e5-3.2e5 photons of the dish, two-mirror, GCT-like and cone
// systems: among photons whose error exceeds 0.3 of the bound, the error stays below 0.87 of the
// estimate, so an unflagged photon stays below 0.78 of the bound (between 0.1 and 0.3 of the
// bound the estimate can fall up to 5% short, far inside it); the largest error of an unflagged
// photon was 0.55 of the bound.
static const double kGuardFrac = 0.9;

// Photons per launch of a source-mode trace with the accuracy guard on: each chunk is followed by
// its own re-trace launch, so the queue (one entry per photon of a chunk) never overflows.
static const long long kSrcChunk = 1LL << 27;

// The feature profile of the kernel that traces g (FP32 or FP64, and the FP32 trace's FP64
// re-trace): a reduced one where it covers the geometry's features (telescopes in plain
// traces, concentrators in either mode), else all.
static unsigned trace_profile(const robast_geom* g, bool src) {
    if (!src && (g->feat & ~(unsigned)FT_TELESCOPE) == 0) return FT_TELESCOPE;
    if ((g->feat & ~(unsigned)FT_CONCENTRATOR) == 0) return FT_CONCENTRATOR;
    return FT_ALL;
}

// The FP64 re-trace of the photons the FP32 launch `a` queued: FP64 arithmetic and tables, the
// FP32 arrays, the same epsilon, random streams and outputs; the queue's length is read on the
// device.
template <typename T>
static cudaError_t launch_retrace_of(const robast_geom* g, robast_geom* gm, const TraceArgs<T>& a,
                                     unsigned long long* qhdr, long long qcap, double eps, bool src, cudaStream_t s) {
    TraceArgs<double, float> r{};
    r.tab = g->tab64;
    r.o = reinterpret_cast<const float*>(a.o);
    r.d = reinterpret_cast<const float*>(a.d);
    r.lam = reinterpret_cast<const float*>(a.lam);
    r.vop = a.vop;
    r.n = a.n;
    r.n_work = qcap;
    r.n_work_dev = qhdr;
    r.queue_in = a.queue_out;
    r.seed = a.seed;
    r.first_id = a.first_id;
    r.max_bounces = a.max_bounces;
    r.refill_min = a.refill_min;
    r.eps = eps;
    r.newton_tol = eps * 1e-4;
    r.newton_tol64 = eps * 1e-4;
    r.st = a.st;
    r.nb = a.nb;
    r.hit = reinterpret_cast<float*>(a.hit);
    r.dir = reinterpret_cast<float*>(a.dir);
    r.last = a.last;
    r.fxy = reinterpret_cast<float*>(a.fxy);
    r.counters = a.counters;
    r.groups = a.groups;
    r.n_groups = a.n_groups;
    r.gcounts = a.gcounts;
    r.err = a.err;
    r.retraced = a.retraced;
    r.work = g->work + (gm->work_slot.fetch_add(1) % kWorkSlots);
    cudaError_t e = cudaMemsetAsync(r.work, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    r.stage = g->smem64 <= kSmemCap ? 1 : 0;
    const size_t smem_r = r.stage ? g->smem64 : 0;
    std::atomic<int>& slot = gm->bps_retrace[src ? 1 : 0];
    int bps_r = slot.load(std::memory_order_relaxed);
    if (bps_r <= 0) {
        bps_r = retrace_blocks_per_sm(smem_r, src, trace_profile(g, src));
        if (bps_r > 0) slot.store(bps_r, std::memory_order_relaxed);
    }
    if (bps_r <= 0) return cudaErrorInvalidConfiguration;
    long long grid_r = (long long)g->num_sms * bps_r;
    grid_r = std::max(1LL, std::min(grid_r, (qcap + 127) / 128));
    return launch_retrace(r, (int)grid_r, smem_r, s, trace_profile(g, src));
}

template <typename T>
static int do_trace(const robast_geom* g, const void* origins, const void* dirs, const void* wl, int64_t n,
                    uint64_t seed, const robast_trace_out* out, const robast_trace_opts& o,
                    const robast_sources* src = nullptr, unsigned long long* gcounts = nullptr) {
    TraceArgs<T> a{};
    if (src) {
        a.groups = src->d_groups;
        a.n_groups = src->n_groups;
        a.gcounts = gcounts;
    }
    a.tab = sizeof(T) == 4 ? g->tab32 : g->tab64;
    a.o = static_cast<const T*>(origins);
    a.d = static_cast<const T*>(dirs);
    a.lam = static_cast<const T*>(wl);
    a.vop = o.variant_of_photon;
    a.n = n;
    a.seed = seed;
    a.first_id = o.first_photon_id;
    a.max_bounces = o.max_bounces;
    if (o.refill_min < 0 || o.refill_min > 32)
        return fail(ROBAST_E_INVALID, "robast_trace: refill_min must be in 0..32 (got %d)", (int)o.refill_min);
    // 24 measured on the dish (refill at 1, 8, 16, 24, 32 idle lanes: 14.0, 11.8, 11.0, 11.0, 11.0 ms)
    a.refill_min = o.refill_min > 0 ? o.refill_min : 24;
    const double L = g->length_scale;
    const double eps = o.eps > 0.0 ? o.eps : (sizeof(T) == 4 ? 1e-6 : 1e-9) * L;
    a.eps = (T)eps;
    // Newton stops at |dt| < 1e-4 eps (FP64: 1e-13 L; FP32: then an FP64 step at grazing incidence)
    a.newton_tol = sizeof(T) == 4 ? (T)(1e-6 * L) : (T)(eps * 1e-4);
    a.newton_tol64 = eps * 1e-4;
    a.st = out->status;
    a.nb = out->bounces;
    a.hit = static_cast<T*>(out->hit);
    a.dir = static_cast<T*>(out->dir);
    a.last = out->last_surface;
    a.fxy = static_cast<T*>(out->focal_xy);
    a.counters = out->counters;
    a.units = o.work_units;
    if (sizeof(T) == 4) a.err = out->err;
    if (!(o.accuracy_pos >= 0.0) || !(o.accuracy_dir >= 0.0))
        return fail(ROBAST_E_INVALID, "robast_trace: accuracy bounds must be >= 0");
    // FP32 accuracy guard: photons over 0.9 of a bound (kGuardFrac) are queued and re-traced in FP64
    const bool guard = sizeof(T) == 4 && (o.accuracy_pos > 0.0 || o.accuracy_dir > 0.0) && !o.track && !o.work_units;
    if (o.track) {
        const robast_track_opts& t = *o.track;
        if (t.first < 0 || t.count < 0 || t.cap < 0 || !t.points || !t.info || !t.n_records)
            return fail(ROBAST_E_INVALID, "robast_trace: track needs first, count, cap >= 0 and device buffers");
        a.tr_first = t.first;
        a.tr_count = t.count;
        a.tr_cap = t.cap;
        a.tr_pts = static_cast<T*>(t.points);
        a.tr_info = t.info;
        a.tr_n = t.n_records;
    }
    cudaStream_t s = static_cast<cudaStream_t>(o.stream);
    robast_geom* gm = const_cast<robast_geom*>(g);
    a.work = g->work + (gm->work_slot.fetch_add(1) % kWorkSlots);
    CU(cudaMemsetAsync(a.work, 0, sizeof(unsigned long long), s), "robast_trace: reset work counter");
    const size_t smem_tab = sizeof(T) == 4 ? g->smem32 : g->smem64;
    a.stage = smem_tab <= kSmemCap ? 1 : 0;
    const size_t smem = a.stage ? smem_tab : 0;
    // default block: 512 for the FP32 kernel (dish: 9.62 ms against 9.88 at 256 and 10.03 at 128;
    // one copy of the staged tables per SM leaves more L1 for the rest), 128 otherwise
    int block = o.block_size ? o.block_size : (sizeof(T) == 4 && !src && !o.work_units ? 512 : 128);
    if (block != 64 && block != 128 && block != 256 && !(block == 512 && sizeof(T) == 4 && !src))
        return fail(ROBAST_E_INVALID, "robast_trace: block_size must be 64, 128 or 256 (or 512 for the FP32 trace; got %d)", block);
    if (a.units && block != 128)
        return fail(ROBAST_E_INVALID, "robast_trace: the counting build (work_units) runs with block_size 128 only");
    if (a.units && src && sizeof(T) != 4)
        return fail(ROBAST_E_INVALID, "robast_trace_sources: the counting build of source mode is FP32 only");
    const int bi = block == 64 ? 0 : block == 128 ? 1 : block == 256 ? 2 : 3;
    std::atomic<int>& bps_slot = gm->bps_cache[sizeof(T) == 4 ? 0 : 1][bi][src ? 1 : 0];
    int bps = bps_slot.load(std::memory_order_relaxed);
    if (bps <= 0) {
        bps = sizeof(T) == 4 ? trace_blocks_per_sm_f32(block, smem, src != nullptr, trace_profile(g, src != nullptr))
                             : trace_blocks_per_sm_f64(block, smem, src != nullptr, trace_profile(g, src != nullptr));
        if (bps > 0) bps_slot.store(bps, std::memory_order_relaxed);
    }
    if (bps <= 0) return fail(ROBAST_E_CUDA, "robast_trace: kernel cannot launch with %zu bytes of shared memory", smem);
    if (o.blocks_per_sm > 0) bps = std::min(bps, (int)o.blocks_per_sm);
    long long grid = (long long)g->num_sms * bps;
    const long long need = (n + block - 1) / block;
    if (grid > need) grid = std::max(1LL, need);
    // coherent processing order (stream-ordered scratch, so concurrent launches do not share it)
    void* ord_scratch = nullptr;
    const bool want_order =
        !src && n > 0 && n < (1LL << 31) && (o.coherent_order > 0 || (o.coherent_order == 0 && n >= 65536));
    if (want_order) {
        CU(cudaMallocFromPoolAsync(&ord_scratch, (size_t)order_scratch_bytes(n), gm->pool, s), "robast_trace: order scratch");
        int* order = nullptr;
        cudaError_t eo;
        if constexpr (sizeof(T) == 4)
            eo = build_order_f32(a.o, n, ord_scratch, &order, g->num_sms, s);
        else
            eo = build_order_f64(a.o, n, ord_scratch, &order, g->num_sms, s);
        if (eo != cudaSuccess) {
            cudaFreeAsync(ord_scratch, s);
            return cuda_fail(eo, "robast_trace: order");
        }
        a.order = order;
    }
    void* q_scratch = nullptr;
    unsigned long long* qhdr = nullptr;
    long long qcap = 0;
    if (guard) {
        if (src) {
            qhdr = src->d_queue;
            qcap = src->qcap;
        } else {
            qcap = n;
            cudaError_t eq = cudaMallocFromPoolAsync(&q_scratch, (size_t)(4 + qcap) * 8, gm->pool, s);
            if (eq != cudaSuccess) {
                if (ord_scratch) cudaFreeAsync(ord_scratch, s);
                return cuda_fail(eq, "robast_trace: re-trace queue");
            }
            qhdr = static_cast<unsigned long long*>(q_scratch);
        }
        cudaError_t eq = cudaMemsetAsync(qhdr, 0, 4 * sizeof(unsigned long long), s);
        if (eq != cudaSuccess) {
            if (ord_scratch) cudaFreeAsync(ord_scratch, s);
            if (q_scratch) cudaFreeAsync(q_scratch, s);
            return cuda_fail(eq, "robast_trace: re-trace queue");
        }
        a.queue_out = reinterpret_cast<long long*>(qhdr + 4);
        a.queue_n = qhdr;
        a.queue_cap = qcap;
        a.acc_pos = o.accuracy_pos > 0.0 ? (float)(kGuardFrac * o.accuracy_pos) : INFINITY;
        a.acc_dir = o.accuracy_dir > 0.0 ? (float)(kGuardFrac * o.accuracy_dir) : INFINITY;
        a.retraced = out->retraced ? out->retraced : qhdr + 1;
    }
    // source mode: each chunk's photons in coherent order, sorted by the cell of their generated
    // origins (the photons of one group and cell share their path, so a warp's lanes and, through
    // the queue's fill order, the FP64 re-trace's stay together)
    const bool src_order = src && src->d_xy && src->d_ord && o.coherent_order >= 0 && !a.units;
    // one launch over all work, or (source mode with the guard or the order) chunks of the source
    // handle's chunk size, each followed by its FP64 re-trace
    const long long chunk = src && (guard || src_order) ? src->qcap : n;
    cudaError_t e = cudaSuccess;
    for (long long base = 0; base < n && e == cudaSuccess; base += chunk) {
        a.work_base = base;
        a.n_work = std::min(chunk, n - base);
        if (base > 0) {
            a.work = g->work + (gm->work_slot.fetch_add(1) % kWorkSlots);
            e = cudaMemsetAsync(a.work, 0, sizeof(unsigned long long), s);
            if (e == cudaSuccess && guard) e = cudaMemsetAsync(qhdr, 0, sizeof(unsigned long long), s);
            if (e != cudaSuccess) break;
        }
        if (src_order) {
            int* order = nullptr;
            e = launch_src_origins(src->d_groups, src->n_groups, base, a.n_work, a.first_id, seed, src->d_xy,
                                   g->num_sms, s);
            if (e == cudaSuccess) e = build_order_f32(src->d_xy, a.n_work, src->d_ord, &order, g->num_sms, s);
            if (e != cudaSuccess) break;
            a.order = order;
        }
        if constexpr (sizeof(T) == 4)
            e = launch_trace_f32(a, block, (int)grid, smem, s, trace_profile(g, src != nullptr));
        else
            e = launch_trace_f64(a, block, (int)grid, smem, s, trace_profile(g, src != nullptr));
        if (e == cudaSuccess && guard) e = launch_retrace_of(g, gm, a, qhdr, qcap, eps, src != nullptr, s);
    }
    if (ord_scratch) cudaFreeAsync(ord_scratch, s);
    if (q_scratch) cudaFreeAsync(q_scratch, s);
    if (e != cudaSuccess) return cuda_fail(e, "robast_trace: launch");
    return 0;
}

static int check_trace_args(const robast_geom* g, const void* o, const void* d, const void* w, int64_t n,
                            const robast_trace_out* out, const robast_trace_opts& op) {
    if (!g) return fail(ROBAST_E_NULL, "robast_trace: geometry is NULL");
    if (!out) return fail(ROBAST_E_NULL, "robast_trace: out is NULL");
    if (n < 0) return fail(ROBAST_E_INVALID, "robast_trace: n must be >= 0 (got %lld)", (long long)n);
    if (n > 0 && (!o || !d || !w)) return fail(ROBAST_E_NULL, "robast_trace: origins, dirs and wavelengths are required");
    if (op.precision != 32 && op.precision != 64)
        return fail(ROBAST_E_INVALID, "robast_trace: precision must be 32 or 64 (got %d)", op.precision);
    if (op.max_bounces < 1 || op.max_bounces > 255)
        return fail(ROBAST_E_INVALID, "robast_trace: max_bounces must be in 1..255 (got %d)", op.max_bounces);
    if (g->n_var > 1 && !op.variant_of_photon && n > 0) {
        // allowed: everything traced through variant 0
    }
    return 0;
}

extern "C" int robast_trace_ex(const robast_geom* g, const void* origins, const void* dirs, const void* wavelengths,
                               int64_t n, uint64_t seed, const robast_trace_out* out, const robast_trace_opts* opts) {
    robast_trace_opts o;
    robast_trace_opts_default(&o);
    if (opts) o = *opts;
    if (o.max_bounces == 0) o.max_bounces = 100;
    if (o.precision == 0) o.precision = 32;
    int rc = check_trace_args(g, origins, dirs, wavelengths, n, out, o);
    if (rc) return rc;
    if (n == 0) return 0;
    return o.precision == 32 ? do_trace<float>(g, origins, dirs, wavelengths, n, seed, out, o)
                             : do_trace<double>(g, origins, dirs, wavelengths, n, seed, out, o);
}

extern "C" int robast_trace(const robast_geom* g, const void* origins, const void* dirs, const void* wavelengths,
                            int64_t n, uint64_t seed, const robast_trace_out* out) {
    return robast_trace_ex(g, origins, dirs, wavelengths, n, seed, out, nullptr);
}

// ---------------------------------------------------------- source groups
extern "C" int robast_sources_create(const robast_geom* g, const robast_source_group* groups, int32_t n_groups,
                                     robast_sources** out) {
    if (!out) return fail(ROBAST_E_NULL, "robast_sources_create: out is NULL");
    *out = nullptr;
    if (!g || !groups) return fail(ROBAST_E_NULL, "robast_sources_create: NULL argument");
    if (n_groups <= 0) return fail(ROBAST_E_INVALID, "robast_sources_create: n_groups must be > 0");
    std::vector<SrcGroup> h(n_groups);
    long long first = 0;
    for (int k = 0; k < n_groups; ++k) {
        const robast_source_group& q = groups[k];
        if (q.variant < 0 || q.variant >= g->n_var)
            return fail(ROBAST_E_INVALID, "robast_sources_create: group %d: variant %d out of range", k, q.variant);
        if (q.n_photons <= 0) return fail(ROBAST_E_INVALID, "robast_sources_create: group %d: n_photons must be > 0", k);
        if (!(q.apothem > 0)) return fail(ROBAST_E_INVALID, "robast_sources_create: group %d: apothem must be > 0", k);
        const double dn = q.dir[0] * q.dir[0] + q.dir[1] * q.dir[1] + q.dir[2] * q.dir[2];
        if (std::fabs(dn - 1.0) > 1e-9) return fail(ROBAST_E_INVALID, "robast_sources_create: group %d: dir not unit", k);
        SrcGroup& G = h[k];
        for (int c = 0; c < 3; ++c) {
            G.c[c] = q.centre[c];
            G.dir[c] = q.dir[c];
        }
        G.a = q.apothem;
        G.R = q.apothem * 2.0 / std::sqrt(3.0);
        G.a32 = (float)G.a;
        G.R32 = (float)G.R;
        G.lam0 = q.lam_min;
        G.lam1 = q.lam_max;
        G.first = first;
        G.n = q.n_photons;
        G.variant = q.variant;
        first += q.n_photons;
    }
    robast_sources* s = new (std::nothrow) robast_sources();
    if (!s) return fail(ROBAST_E_OOM, "robast_sources_create: host allocation failed");
    s->n_groups = n_groups;
    s->n_photons = first;
    s->qcap = std::min<long long>(first, kSrcChunk);
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_groups, h.size() * sizeof(SrcGroup));
    if (e == cudaSuccess) e = cudaMemcpy(s->d_groups, h.data(), h.size() * sizeof(SrcGroup), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_queue, (size_t)(4 + s->qcap) * 8);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_xy, (size_t)s->qcap * 2 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&s->d_ord, (size_t)order_scratch_bytes(s->qcap));
    if (e != cudaSuccess) {
        if (s->d_groups) cudaFree(s->d_groups);
        if (s->d_queue) cudaFree(s->d_queue);
        if (s->d_xy) cudaFree(s->d_xy);
        if (s->d_ord) cudaFree(s->d_ord);
        delete s;
        return cuda_fail(e, "robast_sources_create");
    }
    *out = s;
    return 0;
}

extern "C" void robast_sources_free(robast_sources* s) {
    if (!s) return;
    cudaDeviceSynchronize();
    cudaFree(s->d_groups);
    cudaFree(s->d_queue);
    cudaFree(s->d_xy);
    cudaFree(s->d_ord);
    delete s;
}

extern "C" int robast_sources_info(const robast_sources* s, int32_t* n_groups, int64_t* n_photons) {
    if (!s) return fail(ROBAST_E_NULL, "robast_sources_info: NULL");
    if (n_groups) *n_groups = s->n_groups;
    if (n_photons) *n_photons = s->n_photons;
    return 0;
}

extern "C" int robast_trace_sources(const robast_geom* g, const robast_sources* src, uint64_t seed,
                                    unsigned long long* group_counts, const robast_trace_out* out,
                                    const robast_trace_opts* opts) {
    robast_trace_opts o;
    robast_trace_opts_default(&o);
    if (opts) o = *opts;
    if (o.max_bounces == 0) o.max_bounces = 100;
    if (o.precision == 0) o.precision = 32;
    if (!g || !src) return fail(ROBAST_E_NULL, "robast_trace_sources: NULL geometry or sources");
    if (!group_counts) return fail(ROBAST_E_NULL, "robast_trace_sources: group_counts is required");
    if (o.variant_of_photon) return fail(ROBAST_E_INVALID, "robast_trace_sources: variants come from the groups");
    robast_trace_out none{};
    const robast_trace_out* po = out ? out : &none;
    const char dummy = 0;  // the input pointers are unused in source mode
    int rc = check_trace_args(g, &dummy, &dummy, &dummy, src->n_photons, po, o);
    if (rc) return rc;
    return o.precision == 32 ? do_trace<float>(g, nullptr, nullptr, nullptr, src->n_photons, seed, po, o, src, group_counts)
                             : do_trace<double>(g, nullptr, nullptr, nullptr, src->n_photons, seed, po, o, src, group_counts);
}

static int grow(void** p, size_t* have, size_t need, const char* what) {
    if (*have >= need) return 0;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *have = 0;
    cudaError_t e = cudaMalloc(p, need);
    if (e != cudaSuccess) return fail(ROBAST_E_OOM, "%s: cudaMalloc of %zu bytes failed", what, need);
    *have = need;
    return 0;
}

// pinned host staging: copies from and to it are asynchronous, so a reduction queued
// behind a running trace does not block the host until the trace ends
static int grow_pinned(robast_geom* g, size_t need, const char* what) {
    if (g->pinned_bytes >= need) return 0;
    if (g->pinned) cudaFreeHost(g->pinned);
    g->pinned = nullptr;
    g->pinned_bytes = 0;
    cudaError_t e = cudaMallocHost(&g->pinned, need);
    if (e != cudaSuccess) return fail(ROBAST_E_OOM, "%s: cudaMallocHost of %zu bytes failed", what, need);
    g->pinned_bytes = need;
    return 0;
}

// Host buffers in and out, copies inside.  The photons go in chunks (at least 2^20
// photons, at most 8 chunks) over two internal streams with double-buffered device slices,
// so the upload of chunk c+1 and the download of chunk c-1 overlap the trace of chunk c.
// Photon i keeps id first_photon_id + i, so the results equal one launch over all photons.
extern "C" int robast_trace_host(robast_geom* g, const void* origins, const void* dirs, const void* wavelengths,
                                 int64_t n, uint64_t seed, const robast_trace_out* out, const robast_trace_opts* opts) {
    robast_trace_opts o;
    robast_trace_opts_default(&o);
    if (opts) o = *opts;
    if (o.max_bounces == 0) o.max_bounces = 100;
    if (o.precision == 0) o.precision = 32;
    int rc = check_trace_args(g, origins, dirs, wavelengths, n, out, o);
    if (rc) return rc;
    if (n == 0) return 0;
    std::lock_guard<std::mutex> lk(g->mu);
    const size_t es = o.precision == 32 ? 4 : 8;
    const long long CH = std::max<long long>(1LL << 20, ((long long)n + 7) / 8);  // photons per chunk
    const int nch = (int)((n + CH - 1) / CH);
    const size_t C = (size_t)std::min<long long>(CH, n);
    // one device slice per buffer set (two sets): in o[3C] d[3C] lam[C] vop[C] |
    // out st[C] nb[C] hit[3C] dir[3C] last[C] fxy[2C]; then the counters
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        const size_t at = off;
        off += align16(bytes);
        return at;
    };
    const size_t xo = carve(3 * C * es), xd = carve(3 * C * es), xl = carve(C * es);
    const size_t xv = o.variant_of_photon ? carve(C * 4) : 0;
    const size_t xs = carve(C), xb = carve(C), xh = carve(3 * C * es), xr = carve(3 * C * es), xla = carve(C * 4);
    const size_t xf = carve(2 * C * es);
    const size_t xe = carve(2 * C * 4);
    const size_t set_bytes = off;
    const size_t xc = 2 * set_bytes;
    const int NC = ROBAST_N_COUNTERS + 2;  // the counters, then the accuracy guard's two
    rc = grow(&g->stage, &g->stage_bytes, xc + NC * 8, "robast_trace_host");
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(o.stream);
    for (int k = 0; k < 2; ++k)
        if (!g->hstream[k]) CU(cudaStreamCreateWithFlags(&g->hstream[k], cudaStreamNonBlocking), "robast_trace_host: stream");
    if (!g->hevent) CU(cudaEventCreateWithFlags(&g->hevent, cudaEventDisableTiming), "robast_trace_host: event");
    unsigned char* base = static_cast<unsigned char*>(g->stage);
    unsigned long long* dc = reinterpret_cast<unsigned long long*>(base + xc);
    CU(cudaMemsetAsync(dc, 0, NC * 8, s), "robast_trace_host: counters");
    CU(cudaEventRecord(g->hevent, s), "robast_trace_host: event");  // after the caller's earlier work
    for (int k = 0; k < 2; ++k) CU(cudaStreamWaitEvent(g->hstream[k], g->hevent, 0), "robast_trace_host: wait");
    const unsigned char* ho = static_cast<const unsigned char*>(origins);
    const unsigned char* hd = static_cast<const unsigned char*>(dirs);
    const unsigned char* hl = static_cast<const unsigned char*>(wavelengths);
    const size_t pitch = (size_t)n * es;  // host distance between the x, y, z rows
    for (int c = 0; c < nch; ++c) {
        cudaStream_t st = g->hstream[c & 1];
        unsigned char* b = base + (size_t)(c & 1) * set_bytes;
        const size_t s0 = (size_t)c * CH, nc = (size_t)std::min<long long>(CH, n - (long long)s0);
        // rows of the chunk: x, y, z of photons s0 .. s0 + nc - 1
        CU(cudaMemcpy2DAsync(b + xo, nc * es, ho + s0 * es, pitch, nc * es, 3, cudaMemcpyHostToDevice, st),
           "robast_trace_host: copy in");
        CU(cudaMemcpy2DAsync(b + xd, nc * es, hd + s0 * es, pitch, nc * es, 3, cudaMemcpyHostToDevice, st),
           "robast_trace_host: copy in");
        CU(cudaMemcpyAsync(b + xl, hl + s0 * es, nc * es, cudaMemcpyHostToDevice, st), "robast_trace_host: copy in");
        robast_trace_opts od = o;
        od.stream = st;
        od.first_photon_id = o.first_photon_id + (long long)s0;
        if (o.variant_of_photon) {
            CU(cudaMemcpyAsync(b + xv, o.variant_of_photon + s0, nc * 4, cudaMemcpyHostToDevice, st),
               "robast_trace_host: copy in");
            od.variant_of_photon = reinterpret_cast<const int32_t*>(b + xv);
        }
        robast_trace_out dout{};
        dout.status = out->status ? b + xs : nullptr;
        dout.bounces = out->bounces ? b + xb : nullptr;
        dout.hit = out->hit ? b + xh : nullptr;
        dout.dir = out->dir ? b + xr : nullptr;
        dout.last_surface = out->last_surface ? reinterpret_cast<int32_t*>(b + xla) : nullptr;
        dout.focal_xy = out->focal_xy ? b + xf : nullptr;
        dout.err = out->err && o.precision == 32 ? reinterpret_cast<float*>(b + xe) : nullptr;
        dout.counters = dc;
        dout.retraced = dc + ROBAST_N_COUNTERS;
        rc = robast_trace_ex(g, b + xo, b + xd, b + xl, (int64_t)nc, seed, &dout, &od);
        if (rc) return rc;
        unsigned char* os = static_cast<unsigned char*>(out->status);
        unsigned char* ob = static_cast<unsigned char*>(out->bounces);
        unsigned char* oh = static_cast<unsigned char*>(out->hit);
        unsigned char* orr = static_cast<unsigned char*>(out->dir);
        unsigned char* ol = reinterpret_cast<unsigned char*>(out->last_surface);
        unsigned char* of = static_cast<unsigned char*>(out->focal_xy);
        if (os) CU(cudaMemcpyAsync(os + s0, dout.status, nc, cudaMemcpyDeviceToHost, st), "copy out");
        if (ob) CU(cudaMemcpyAsync(ob + s0, dout.bounces, nc, cudaMemcpyDeviceToHost, st), "copy out");
        if (oh) CU(cudaMemcpy2DAsync(oh + s0 * es, pitch, dout.hit, nc * es, nc * es, 3, cudaMemcpyDeviceToHost, st), "copy out");
        if (orr) CU(cudaMemcpy2DAsync(orr + s0 * es, pitch, dout.dir, nc * es, nc * es, 3, cudaMemcpyDeviceToHost, st), "copy out");
        if (ol) CU(cudaMemcpyAsync(ol + s0 * 4, dout.last_surface, nc * 4, cudaMemcpyDeviceToHost, st), "copy out");
        if (of) CU(cudaMemcpy2DAsync(of + s0 * es, pitch, dout.focal_xy, nc * es, nc * es, 2, cudaMemcpyDeviceToHost, st), "copy out");
        if (dout.err)
            CU(cudaMemcpy2DAsync(reinterpret_cast<unsigned char*>(out->err) + s0 * 4, (size_t)n * 4, dout.err, nc * 4,
                                 nc * 4, 2, cudaMemcpyDeviceToHost, st), "copy out");
    }
    unsigned long long hc[NC];
    for (int k = 0; k < 2; ++k) CU(cudaStreamSynchronize(g->hstream[k]), "robast_trace_host: synchronize");
    CU(cudaMemcpy(hc, dc, sizeof hc, cudaMemcpyDeviceToHost), "copy out");
    if (out->counters)
        for (int k = 0; k < ROBAST_N_COUNTERS; ++k) out->counters[k] += hc[k];
    if (out->retraced)
        for (int k = 0; k < 2; ++k) out->retraced[k] += hc[ROBAST_N_COUNTERS + k];
    return 0;
}

// -------------------------------------------------------------- gradients
extern "C" int robast_param_count(const robast_geom* g) { return g ? g->n_surf * ROBAST_N_PARAM : 0; }

extern "C" int robast_param_layout(const robast_geom* g, robast_param_info* out) {
    if (!g || !out) return fail(ROBAST_E_NULL, "robast_param_layout: NULL argument");
    for (int s = 0; s < g->n_surf; ++s) {
        const int shape = g->h_flags[s] & 15, role = (g->h_flags[s] >> 4) & 15;
        const bool mirror = role == ROBAST_ROLE_MIRROR;
        for (int k = 0; k < ROBAST_N_PARAM; ++k) {
            robast_param_info& p = out[(size_t)s * ROBAST_N_PARAM + k];
            p.surface = s;
            p.variant = g->h_var[s];
            p.slot = k;
            // the gradient pass differentiates SAG mirrors (tilts, A1..A8) and HEXCONE mirrors (Bezier points)
            p.active = mirror && ((shape == ROBAST_SHAPE_SAG && k < 10) || (shape == ROBAST_SHAPE_HEXCONE && k >= 10));
        }
    }
    return 0;
}

template <typename T>
static int do_grad(robast_geom* g, const void* o, const void* d, const void* wl, int64_t n, uint64_t seed,
                   int objective, double tau, double d_obj, double* value, double* d_params,
                   const robast_trace_opts& op, double* info) {
    GradArgs<T> a{};
    a.tab = sizeof(T) == 4 ? g->tab32 : g->tab64;
    a.surf64 = static_cast<const double*>(g->tab64.surf);
    a.grec = g->grec64;
    a.o = static_cast<const T*>(o);
    a.d = static_cast<const T*>(d);
    a.lam = static_cast<const T*>(wl);
    a.vop = op.variant_of_photon;
    a.n = n;
    a.seed = seed;
    a.first_id = op.first_photon_id;
    a.max_bounces = op.max_bounces;
    const double L = g->length_scale;
    const double eps = op.eps > 0.0 ? op.eps : (sizeof(T) == 4 ? 1e-6 : 1e-9) * L;
    a.eps = (T)eps;
    a.newton_tol = sizeof(T) == 4 ? (T)(1e-6 * L) : (T)(eps * 1e-4);
    a.newton_tol64 = 1e-13 * L;
    a.objective = objective;
    a.tau = tau;
    a.units = op.work_units;  // the gradient pass's three work units, when asked for
    const size_t NP = (size_t)g->n_surf * ROBAST_N_PARAM;
    const size_t NV = (size_t)g->n_var;
    std::lock_guard<std::mutex> lk(g->mu);
    // 128-bit fixed-point sums: GRAD_SLOTS words per surface, 16 per variant
    const size_t words = (size_t)g->n_surf * GRAD_SLOTS + 16 * NV;
    int rc = grow(&g->scratch, &g->scratch_bytes, words * 8, "robast_trace_grad");
    if (rc) return rc;
    unsigned long long* acc = static_cast<unsigned long long*>(g->scratch);
    unsigned long long* vals = acc + (size_t)g->n_surf * GRAD_SLOTS;
    a.acc = acc;
    a.vals = vals;
    cudaStream_t s = static_cast<cudaStream_t>(op.stream);
    CU(cudaMemsetAsync(acc, 0, words * 8, s), "robast_trace_grad: clear");
    const size_t smem_tab = sizeof(T) == 4 ? g->smem32 : g->smem64;
    a.stage = smem_tab <= kSmemCap ? 1 : 0;
    const size_t smem = a.stage ? smem_tab : 0;
    // derivative passes in FP32 for an FP32 trace, except through Bezier cone walls (their grazing
    // roots need FP64); one resident wave: the kernel strides over the photons
    const bool r64 = sizeof(T) == 8 || (g->feat & FT_CONE) != 0;
    const int bps = sizeof(T) == 8 ? grad_blocks_per_sm_f64(smem)
                    : r64          ? grad_blocks_per_sm_f32_r64(smem)
                                   : grad_blocks_per_sm_f32(smem);
    if (bps <= 0) return fail(ROBAST_E_CUDA, "robast_trace_grad: the gradient kernel cannot launch with %zu bytes of shared memory", smem);
    const long long grid = std::max(1LL, std::min<long long>((long long)g->num_sms * bps, (n + 127) / 128));
    // coherent processing order (stream-ordered scratch from g's pool).  By default only for
    // geometries with cones, where a path's wall reflections diverge most (soft-CE gradient
    // 248 -> 142 ms per 1e6 photons).  On a dish batch the coherent order raises the active lanes
    // but the kernel then waits far longer on instruction fetch (its code and spilled frames;
    // MSR gradient 144 -> 213 ms per 3.2e7 photons), so id order stays the default there
    void* ord_scratch = nullptr;
    const bool want_order = op.coherent_order > 0 || (op.coherent_order == 0 && n >= 65536 && (g->feat & FT_CONE) != 0);
    if (n > 0 && n < (1LL << 31) && want_order) {
        CU(cudaMallocFromPoolAsync(&ord_scratch, (size_t)order_scratch_bytes(n), g->pool, s),
           "robast_trace_grad: order scratch");
        int* order = nullptr;
        cudaError_t eo;
        if constexpr (sizeof(T) == 4)
            eo = build_order_f32(a.o, n, ord_scratch, &order, g->num_sms, s);
        else
            eo = build_order_f64(a.o, n, ord_scratch, &order, g->num_sms, s);
        if (eo != cudaSuccess) {
            cudaFreeAsync(ord_scratch, s);
            return cuda_fail(eo, "robast_trace_grad: order");
        }
        a.order = order;
    }
    cudaError_t e;
    if constexpr (sizeof(T) == 4)
        e = r64 ? launch_grad_f32_r64(a, (int)grid, smem, s) : launch_grad_f32(a, (int)grid, smem, s);
    else
        e = launch_grad_f64(a, (int)grid, smem, s);
    if (ord_scratch) cudaFreeAsync(ord_scratch, s);
    if (e != cudaSuccess) return cuda_fail(e, "robast_trace_grad: launch");
    if (d_params) {
        e = launch_grad_finish(acc, vals, g->surf_var, (int)NP, objective, d_obj, d_params, s);
        if (e != cudaSuccess) return cuda_fail(e, "robast_trace_grad: launch");
    }
    std::vector<unsigned long long> hw(16 * NV);
    CU(cudaMemcpyAsync(hw.data(), vals, hw.size() * 8, cudaMemcpyDeviceToHost, s), "robast_trace_grad: copy");
    CU(cudaStreamSynchronize(s), "robast_trace_grad: synchronize");
    std::vector<double> hv(8 * NV);
    for (size_t k = 0; k < hv.size(); ++k) hv[k] = grad_fx_value(&hw[2 * k]);
    // the objective of several variants is the sum of their objectives
    double total = 0.0;
    for (size_t v = 0; v < NV; ++v) {
        const double* V = &hv[8 * v];
        if (objective == 1) {
            if (V[7] > 0) total += V[4] / V[7];
        } else if (V[0] > 0) {
            const double qx = V[1] / V[0], qy = V[2] / V[0];
            if (objective == 0) total += V[3] / V[0] - qx * qx - qy * qy;
            if (objective == 2) total += qx;
            if (objective == 3) total += qy;
        }
    }
    *value = total;
    if (info) {
        for (int k = 0; k < 8; ++k) info[k] = 0.0;
        for (size_t v = 0; v < NV; ++v)
            for (int k = 0; k < 8; ++k) info[k] += hv[8 * v + k];
    }
    return 0;
}

extern "C" int robast_trace_grad(robast_geom* g, const void* origins, const void* dirs, const void* wavelengths,
                                 int64_t n, uint64_t seed, int32_t objective, double tau, double d_obj, double* value,
                                 double* d_params, const robast_trace_opts* opts, double* info) {
    robast_trace_opts o;
    robast_trace_opts_default(&o);
    if (opts) o = *opts;
    if (o.max_bounces == 0) o.max_bounces = 100;
    if (o.precision == 0) o.precision = 32;
    if (!value) return fail(ROBAST_E_NULL, "robast_trace_grad: value is NULL");
    robast_trace_out none{};
    int rc = check_trace_args(g, origins, dirs, wavelengths, n, &none, o);
    if (rc) return rc;
    if (n <= 0) return fail(ROBAST_E_INVALID, "robast_trace_grad: n must be > 0");
    if (objective < 0 || objective > 3) return fail(ROBAST_E_INVALID, "robast_trace_grad: unknown objective %d", objective);
    if (objective == 1 && !(tau > 0.0)) return fail(ROBAST_E_INVALID, "robast_trace_grad: tau must be > 0");
    robast_geom* gm = const_cast<robast_geom*>(g);
    return o.precision == 32 ? do_grad<float>(gm, origins, dirs, wavelengths, n, seed, objective, tau, d_obj, value,
                                              d_params, o, info)
                             : do_grad<double>(gm, origins, dirs, wavelengths, n, seed, objective, tau, d_obj, value,
                                               d_params, o, info);
}

// ------------------------------------------------------------- reductions
// Spot diagrams of several photon windows at once.  Per window: centroid
// from fixed-order block partials; R80 = exact nearest-rank 80th percentile
// of the radius to the centroid.  Ordering by r^2 is ordering by r, and r =
// sqrt(r^2) of the selected photon, so no square root or division is taken
// per photon.  The rank is located on the device in two histogram rounds:
//   1. r^2 over [0, (8 x RMS radius)^2) in kBins bins plus an overflow bin;
//      the bins lo..hi around the bin b that holds the rank are kept;
//   2. the exact FP64 r^2 of the photons kept, in kSub sub-bins of an
//      interval that covers them (indices clamped, so the sub-bin is a
//      non-decreasing function of r^2 whatever the interval);
// then the values of the sub-bin that holds the rank (a handful) are
// collected and the rank is selected among them by counting.  One host
// synchronisation per call; a sub-bin with more than kSel distinct values
// (a spot far more concentrated than its RMS radius suggests) falls back to
// collecting bins lo..hi and selecting on the host.
//
// FP64 issues at a small fraction of the FP32 rate on this GPU, so with FP32
// positions the first round takes no FP64 operation per photon: the sums are
// float pairs, and the histogram bins an FP32 r^2 whose error, in bins, is
// bounded by delta in psf_finish.  When delta < 1/2, every photon outside the
// bins b-1..b+1 lies on the correct side of the rank photon in exact
// arithmetic (approximate and exact bin positions differ by at most delta),
// so lo..hi = b-1..b+1 holds the rank photon and the photons below lo are
// exactly those ranked below the kept ones.  Otherwise (a spot tiny against
// its distance from the origin) the window is binned in FP64 and lo = hi = b.
namespace {
constexpr int kRedBlock = 256;
constexpr int kPartBlocks = 1216;  // blocks of a per-photon pass over all windows (8 per SM)
constexpr int kBins = 4096;        // + 1 overflow bin
constexpr int kSub = 4096;         // second-round sub-bins
constexpr int kSel = 2048;         // values the device selects among
constexpr int kScanBlock = 1024;
constexpr int kRes = 8;            // per window: N, cx, cy, bins / range^2, fast, delta, -, -
constexpr int kUnroll = 4;         // photons in flight per thread
constexpr long long kCandPerWindow = 1LL << 20;  // candidate list capacity per window
constexpr long long kCandTotal = 1LL << 23;      // ... and over all windows of a call
namespace cg = cooperative_groups;

// blocks per window of the per-photon passes (robast_psf and robast_psf_noalloc alike)
int psf_blocks_per_window(int nw, long long maxcount) {
    return (int)std::max(1LL, std::min<long long>(std::max(1, kPartBlocks / nw), (maxcount + kRedBlock - 1) / kRedBlock));
}

struct Win {
    long long start, count;
    long long cand_off, cand_slice;  // this window's part of the candidate list: one slice per block (robast_psf)
};

// unevaluated float pair hi + lo; two-sum (Knuth) keeps every addition exact
// in the pair, the product error comes from a fused multiply-add (Dekker)
struct F2 {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float s = __fadd_rn(hi, x);
        const float bp = __fsub_rn(s, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
        hi = s;
        lo = __fadd_rn(lo, e);
    }
    __device__ __forceinline__ void add_sq(float x) {
        const float p = __fmul_rn(x, x);
        add(p);
        lo = __fadd_rn(lo, __fmaf_rn(x, x, -p));
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Per-thread partial sums over photons start + k, k = tid, tid + stride, ...:
// (detected count, sum x, sum y, sum x^2, sum y^2), loads kUnroll photons
// ahead.  Shared by robast_psf and robast_psf_noalloc, so their centroids
// agree bit for bit.
__device__ __forceinline__ void psf_thread_sums(const uint8_t* st, const float* fxy, long long ld, long long start,
                                                long long count, long long tid, long long stride, double out[5]) {
    unsigned n = 0;
    F2 sx, sy, sxx, syy;
    for (long long k0 = tid; k0 < count; k0 += kUnroll * stride) {
        uint8_t s[kUnroll];
        float x[kUnroll], y[kUnroll];
#pragma unroll
        for (int j = 0; j < kUnroll; ++j) {
            const long long k = k0 + j * stride;
            s[j] = 0;
            x[j] = y[j] = 0.0f;
            if (k < count) {
                s[j] = st[start + k];
                x[j] = fxy[start + k];
                y[j] = fxy[ld + start + k];
            }
        }
#pragma unroll
        for (int j = 0; j < kUnroll; ++j)
            if (s[j] == ROBAST_ST_DETECTED) {
                ++n;
                sx.add(x[j]);
                sy.add(y[j]);
                sxx.add_sq(x[j]);
                syy.add_sq(y[j]);
            }
    }
    out[0] = (double)n;
    out[1] = sx.value();
    out[2] = sy.value();
    out[3] = sxx.value();
    out[4] = syy.value();
}

__device__ __forceinline__ void psf_thread_sums(const uint8_t* st, const double* fxy, long long ld, long long start,
                                                long long count, long long tid, long long stride, double out[5]) {
    double acc[5] = {0, 0, 0, 0, 0};
    for (long long k = tid; k < count; k += stride) {
        const long long i = start + k;
        if (st[i] == ROBAST_ST_DETECTED) {
            const double x = fxy[i], y = fxy[ld + i];
            acc[0] += 1.0;
            acc[1] += x;
            acc[2] += y;
            acc[3] += x * x;
            acc[4] += y * y;
        }
    }
    for (int c = 0; c < 5; ++c) out[c] = acc[c];
}

template <typename T>
__global__ void psf_sums(const uint8_t* st, const T* fxy, long long ld, const Win* win, double* part) {
    const Win w = win[blockIdx.y];
    double acc[5];
    psf_thread_sums(st, fxy, ld, w.start, w.count, blockIdx.x * (long long)blockDim.x + threadIdx.x,
                    (long long)gridDim.x * blockDim.x, acc);
    __shared__ double sh[5][kRedBlock];
    for (int c = 0; c < 5; ++c) sh[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int h = kRedBlock / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int c = 0; c < 5; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 5; ++c) part[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 5 + c] = sh[c][0];
}

// Window sums from the block partials in a fixed order: lane l adds the
// partials l, l + 32, ... in turn, then a butterfly (each step adds the same
// two numbers on both lanes, so all lanes end with the same bits).  One full
// warp per window; robast_psf and robast_psf_noalloc share it, so their
// centroids agree bit for bit.
__device__ __forceinline__ void psf_window_sums(const double* part, int nblocks, int w, double a[5]) {
    const int lane = threadIdx.x & 31;
    for (int c = 0; c < 5; ++c) a[c] = 0.0;
    for (int b = lane; b < nblocks; b += 32)
        for (int c = 0; c < 5; ++c) a[c] += part[((size_t)w * nblocks + b) * 5 + c];
    for (int off = 16; off > 0; off >>= 1)
        for (int c = 0; c < 5; ++c) a[c] += __shfl_xor_sync(0xffffffffu, a[c], off);
}

// One warp per window.  res = (N, cx, cy, bins / range^2, fast, delta).
// delta bounds |approximate - exact| bin position of the FP32 binning
// (psf_fbin) for every photon with exact r^2 < (kBins + 2) / scale; fast = 1
// when FP32 binning may be used.
__global__ void psf_finish(const double* part, int nblocks, int allow_fast, double* res) {
    const int w = blockIdx.x;
    double a[5];
    psf_window_sums(part, nblocks, w, a);
    if (threadIdx.x != 0) return;
    const double n = a[0];
    const double cx = n > 0 ? a[1] / n : 0.0, cy = n > 0 ? a[2] / n : 0.0;
    const double ms = n > 0 ? fmax(0.0, (a[3] + a[4]) / n - cx * cx - cy * cy) : 0.0;
    const double range2 = fmax(64.0 * ms, 1e-300);  // (8 x RMS radius)^2
    const double scale = (double)kBins / range2;
    // Error of psf_fbin for |dx|, |dy| <= R (u = unit roundoff of FP32):
    //   dxf = fl(x - fl(cx)) differs from x - cx by ex <= u|cx|(1+u) + uR,
    //   |dxf^2 - dx^2| <= ex(2R + ex), the fma and product add (2u+u^2) E^2
    //   with E = R + ex + ey, and the scaling by fl(scale) another (2u+u^2).
    const double u = 0x1p-24, R2 = (kBins + 2) / scale, R = sqrt(R2);
    const double ex = u * fabs(cx) * (1 + u) + u * R, ey = u * fabs(cy) * (1 + u) + u * R;
    const double E = R + ex + ey;
    const double err = ex * (2 * R + ex) + ey * (2 * R + ey) + (2 * u + u * u) * E * E;
    const double delta = scale * err + (2 * u + u * u) * scale * (R2 + err);
    const bool fast = allow_fast && n > 0 && scale < 1e37 && fabs(cx) < 1e37 && fabs(cy) < 1e37 &&
                      1.5 * delta < 0.25;  // margin of 2 against the bound 1/2
    double* r = res + kRes * w;
    r[0] = n;
    r[1] = cx;
    r[2] = cy;
    r[3] = scale;
    r[4] = fast ? 1.0 : 0.0;
    r[5] = delta;
    r[6] = r[7] = 0.0;
}

// exact bin of r^2: scale = kBins / range^2; values beyond the range -> overflow bin
__device__ __forceinline__ int psf_bin(double r2, double scale) {
    const double f = r2 * scale;
    if (!(f < (double)kBins)) return kBins;
    const int b = (int)f;
    return b < 0 ? 0 : b;
}

// approximate bin in FP32, each rounding explicit (the error bound above
// follows these operations)
__device__ __forceinline__ int psf_fbin(float x, float y, float cx, float cy, float scale) {
    const float dx = __fsub_rn(x, cx), dy = __fsub_rn(y, cy);
    const float f = __fmul_rn(__fmaf_rn(dx, dx, __fmul_rn(dy, dy)), scale);
    if (!(f < (float)kBins)) return kBins;
    return (int)f;
}

template <typename T>
__device__ __forceinline__ double psf_r2(T x, T y, const double* R) {
    const double dx = (double)x - R[1], dy = (double)y - R[2];
    return dx * dx + dy * dy;
}

// Bin of each photon of one window, kUnroll photons in flight per thread;
// body(bin, x, y, i) runs for the detected ones (i: photon index).  FAST:
// FP32 bins (psf_fbin).
template <bool FAST, typename T, typename F>
__device__ __forceinline__ void psf_loop(const uint8_t* st, const T* fxy, long long ld, const Win& w, const double* R,
                                         F body) {
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
    const float cxf = __double2float_rn(R[1]), cyf = __double2float_rn(R[2]), sf = __double2float_rn(R[3]);
    for (long long k0 = tid; k0 < w.count; k0 += kUnroll * stride) {
        uint8_t s[kUnroll];
        T x[kUnroll], y[kUnroll];
#pragma unroll
        for (int j = 0; j < kUnroll; ++j) {
            const long long k = k0 + j * stride;
            s[j] = 0;
            x[j] = y[j] = T(0);
            if (k < w.count) {
                s[j] = st[w.start + k];
                x[j] = fxy[w.start + k];
                y[j] = fxy[ld + w.start + k];
            }
        }
#pragma unroll
        for (int j = 0; j < kUnroll; ++j)
            if (s[j] == ROBAST_ST_DETECTED) {
                int b;
                if constexpr (FAST)
                    b = psf_fbin((float)x[j], (float)y[j], cxf, cyf, sf);
                else
                    b = psf_bin(psf_r2(x[j], y[j], R), R[3]);
                body(b, x[j], y[j], w.start + k0 + j * stride);
            }
    }
}

// The window's binning is chosen once per block (a uniform branch), so the
// FP32 loop carries no FP64 operation.
template <typename T, typename F>
__device__ __forceinline__ void psf_for_bins(const uint8_t* st, const T* fxy, long long ld, const Win& w,
                                             const double* R, F body) {
    if constexpr (sizeof(T) == 4) {
        if (R[4] != 0.0) {
            psf_loop<true>(st, fxy, ld, w, R, body);
            return;
        }
    }
    psf_loop<false>(st, fxy, ld, w, R, body);
}

// sub-bin of r^2 in the second histogram (non-decreasing in r^2 for any a and s2 >= 0)
__device__ __forceinline__ int psf_sub(double r2, double a, double s2) {
    const double f = (r2 - a) * s2;
    if (!(f > 0.0)) return 0;  // also NaN
    return f >= (double)kSub ? kSub - 1 : (int)f;
}

template <typename T>
__global__ void psf_hist(const uint8_t* st, const T* fxy, long long ld, const Win* win, const double* res,
                         unsigned long long* hist) {
    __shared__ unsigned int h[kBins + 1];
    for (int k = threadIdx.x; k <= kBins; k += blockDim.x) h[k] = 0;
    __syncthreads();
    const Win w = win[blockIdx.y];
    psf_for_bins(st, fxy, ld, w, res + kRes * blockIdx.y, [&](int b, T, T, long long) { atomicAdd(&h[b], 1u); });
    __syncthreads();
    unsigned long long* H = hist + (size_t)blockIdx.y * (kBins + 1);
    for (int k = threadIdx.x; k <= kBins; k += blockDim.x)
        if (h[k]) atomicAdd(H + k, (unsigned long long)h[k]);
}

// Fallback selection: the values of bins lo..hi.  sel[4w..] = (first bin,
// last bin, offset into vals, -); cnt[w] counts the values written; each
// value is the photon's exact FP64 r^2.
template <typename T>
__global__ void psf_collect(const uint8_t* st, const T* fxy, long long ld, const Win* win, const double* res,
                            const long long* sel, double* vals, unsigned long long* cnt, const long long* cap) {
    const Win w = win[blockIdx.y];
    const double* R = res + kRes * blockIdx.y;
    const int lo = (int)sel[4 * blockIdx.y], hi = (int)sel[4 * blockIdx.y + 1];
    double* out = vals + sel[4 * blockIdx.y + 2];
    const long long c = cap[blockIdx.y];
    unsigned long long* cw = cnt + blockIdx.y;
    psf_for_bins(st, fxy, ld, w, R, [&](int b, T x, T y, long long) {
        if (b >= lo && b <= hi) {
            const unsigned long long j = atomicAdd(cw, 1ull);
            if ((long long)j < c) out[j] = psf_r2(x, y, R);
        }
    });
}

// Device-side selection state of one window.
struct Sel {
    long long k;      // rank of the 80% photon among the window's detected photons
    long long rank1;  // its rank among the photons of first-round bins lo..hi
    long long cap1;   // photons in bins lo..hi
    long long rank2;  // its rank among the values of sub-bin sub
    long long cap2;   // values in sub-bin sub
    double a, s2;     // sub-bin of r^2: clamp(floor((r^2 - a) s2), 0, kSub - 1)
    int lo, hi;       // first-round bins kept
    int sub;          // chosen sub-bin
    int status;       // 0 in progress / resolved, 1 unresolved, 2 no detected photon, 3 counts disagree
};

// Block of kScanBlock threads: the bin j of H[0..nb) with
// sum(H[0..j)) <= k < sum(H[0..j]) (-1 if k >= total), sum(H[0..j)) and the
// total, to every thread.
__device__ void block_find_rank(const unsigned long long* H, int nb, long long k, int* bin, long long* below,
                                long long* total) {
    __shared__ unsigned long long csum[kScanBlock];
    __shared__ int s_bin;
    __shared__ long long s_below;
    const int per = (nb + kScanBlock - 1) / kScanBlock;
    const int j0 = min(nb, (int)threadIdx.x * per), j1 = min(nb, j0 + per);
    unsigned long long my = 0;
    for (int j = j0; j < j1; ++j) my += H[j];
    csum[threadIdx.x] = my;
    if (threadIdx.x == 0) {
        s_bin = -1;
        s_below = 0;
    }
    __syncthreads();
    for (int off = 1; off < kScanBlock; off <<= 1) {  // inclusive scan
        const unsigned long long v = (int)threadIdx.x >= off ? csum[threadIdx.x - off] : 0ull;
        __syncthreads();
        csum[threadIdx.x] += v;
        __syncthreads();
    }
    const long long before = (long long)(csum[threadIdx.x] - my);
    if (before <= k && k < before + (long long)my) {  // one thread at most
        long long acc = before;
        for (int j = j0; j < j1; ++j) {
            if (acc + (long long)H[j] > k) {
                s_bin = j;
                s_below = acc;
                break;
            }
            acc += (long long)H[j];
        }
    }
    __syncthreads();
    *bin = s_bin;
    *below = s_below;
    *total = (long long)csum[kScanBlock - 1];
}

// First-histogram decision: rank k, bin b, bins lo..hi kept, the sub-bin interval.
__global__ void psf_pick1(const unsigned long long* hist, const double* res, const Win* win, int nslice, Sel* sel) {
    const int w = blockIdx.x;
    const double* R = res + kRes * w;
    const long long N = (long long)R[0];
    Sel z{};
    z.k = -1;
    z.lo = -1;
    z.hi = -2;
    z.sub = -1;
    if (N == 0) {
        if (threadIdx.x == 0) {
            z.status = 2;
            sel[w] = z;
        }
        return;
    }
    const long long k = (long long)ceil(0.8 * (double)N) - 1;
    const unsigned long long* H = hist + (size_t)w * (kBins + 1);
    int b;
    long long below, total;
    block_find_rank(H, kBins + 1, k, &b, &below, &total);
    if (threadIdx.x != 0) return;
    z.k = k;
    if (b < 0 || total != N) {
        z.status = 3;
        sel[w] = z;
        return;
    }
    const bool fast = R[4] != 0.0;
    const int lo = fast ? max(b - 1, 0) : b, hi = fast ? min(b + 1, kBins) : b;
    long long below1 = below, cap1 = 0;
    for (int j = lo; j < b; ++j) below1 -= (long long)H[j];
    for (int j = lo; j <= hi; ++j) cap1 += (long long)H[j];
    z.lo = lo;
    z.hi = hi;
    z.rank1 = k - below1;
    z.cap1 = cap1;
    if (cap1 > win[w].cand_slice * nslice) {  // more kept photons than the candidate list holds: host fallback
        z.status = 1;
        sel[w] = z;
        return;
    }
    // exact r^2 of the kept photons lies in [(lo - delta) / scale, (hi + 1 + delta) / scale]
    const double scale = R[3];
    z.a = fmax(0.0, ((double)lo - 0.5) / scale);
    z.s2 = (double)kSub / (((double)hi + 1.5) / scale - z.a);
    z.status = 0;
    sel[w] = z;
}

// Compaction: the index of every kept photon (bins lo..hi) appended to the
// block's slice of the window's candidate list (a counter per block, one
// atomic per group of lanes that keep one).  Only FP32 work per photon; the
// kept photons' FP64 r^2 follows over the short list, where every lane of a
// warp has one.
template <typename T>
__global__ void psf_compact(const uint8_t* st, const T* fxy, long long ld, const Win* win, const double* res,
                            const Sel* sel, long long* cand, unsigned long long* cand_n) {
    const Win w = win[blockIdx.y];
    const Sel S = sel[blockIdx.y];
    if (S.status != 0) return;
    long long* out = cand + w.cand_off + blockIdx.x * w.cand_slice;
    unsigned long long* cn = cand_n + (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    psf_for_bins(st, fxy, ld, w, res + kRes * blockIdx.y, [&](int b, T, T, long long i) {
        if (b >= S.lo && b <= S.hi) {
            cg::coalesced_group g = cg::coalesced_threads();
            unsigned long long base = 0;
            if (g.thread_rank() == 0) base = atomicAdd(cn, (unsigned long long)g.size());
            base = g.shfl(base, 0);
            const unsigned long long j = base + g.thread_rank();
            if ((long long)j < w.cand_slice) out[j] = i;
        }
    });
}

// One warp per window: a slice that overflowed sends the window to the host
// fallback; otherwise the slices must hold exactly the cap1 kept photons.
__global__ void psf_cand_check(const Win* win, const unsigned long long* cand_n, int nslice, Sel* sel) {
    const int w = blockIdx.x;
    if (sel[w].status != 0) return;
    unsigned long long tot = 0;
    int over = 0;
    for (int b = threadIdx.x; b < nslice; b += 32) {
        const unsigned long long c = cand_n[(size_t)w * nslice + b];
        tot += c;
        over |= c > (unsigned long long)win[w].cand_slice;
    }
    for (int off = 16; off > 0; off >>= 1) {
        tot += __shfl_xor_sync(0xffffffffu, tot, off);
        over |= __shfl_xor_sync(0xffffffffu, over, off);
    }
    if (threadIdx.x == 0) sel[w].status = over ? 1 : ((long long)tot != sel[w].cap1 ? 3 : 0);
}

// Entry t of the window's candidate list (slice t / cand_slice), if filled.
__device__ __forceinline__ bool psf_cand_at(const Win& w, const unsigned long long* cn, long long t) {
    const long long b = t / w.cand_slice, j = t - b * w.cand_slice;
    return j < (long long)cn[b];
}

// The kept photons' exact FP64 r^2, over the candidate list.
template <typename T>
__global__ void psf_cand_r2(const T* fxy, long long ld, const Win* win, const double* res, const Sel* sel,
                            const long long* cand, const unsigned long long* cand_n, int nslice, double* r2) {
    const Sel S = sel[blockIdx.y];
    if (S.status != 0) return;
    const Win w = win[blockIdx.y];
    const double* R = res + kRes * blockIdx.y;
    const unsigned long long* cn = cand_n + (size_t)blockIdx.y * nslice;
    const long long n = w.cand_slice * nslice;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        if (psf_cand_at(w, cn, t)) {
            const long long i = cand[w.cand_off + t];
            r2[w.cand_off + t] = psf_r2(fxy[i], fxy[ld + i], R);
        }
}

// Second histogram: sub-bins of the kept photons' exact r^2.
__global__ void psf_hist2(const Win* win, const Sel* sel, const double* r2, const unsigned long long* cand_n,
                          int nslice, unsigned long long* hist2) {
    __shared__ unsigned int h[kSub];
    for (int k = threadIdx.x; k < kSub; k += blockDim.x) h[k] = 0;
    __syncthreads();
    const Sel S = sel[blockIdx.y];
    const Win w = win[blockIdx.y];
    if (S.status == 0) {
        const unsigned long long* cn = cand_n + (size_t)blockIdx.y * nslice;
        const long long n = w.cand_slice * nslice;
        for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
            if (psf_cand_at(w, cn, t)) atomicAdd(&h[psf_sub(r2[w.cand_off + t], S.a, S.s2)], 1u);
    }
    __syncthreads();
    unsigned long long* H = hist2 + (size_t)blockIdx.y * kSub;
    for (int k = threadIdx.x; k < kSub; k += blockDim.x)
        if (h[k]) atomicAdd(H + k, (unsigned long long)h[k]);
}

// Second-histogram decision: the sub-bin that holds rank1.
__global__ void psf_pick2(const unsigned long long* hist2, Sel* sel) {
    const int w = blockIdx.x;
    const Sel S = sel[w];
    if (S.status != 0) return;
    const unsigned long long* H = hist2 + (size_t)w * kSub;
    int sub;
    long long below, total;
    block_find_rank(H, kSub, S.rank1, &sub, &below, &total);
    if (threadIdx.x != 0) return;
    if (sub < 0 || total != S.cap1) {
        sel[w].status = 3;
        return;
    }
    sel[w].sub = sub;
    sel[w].rank2 = S.rank1 - below;
    sel[w].cap2 = (long long)H[sub];
}

// The exact r^2 of the sub-bin's photons (at most kSel kept), their count
// and the bit patterns of their minimum (stored complemented) and maximum.
__global__ void psf_collect2(const Win* win, const Sel* sel, const double* r2, const unsigned long long* cand_n,
                             int nslice, double* vals2, unsigned long long* cnt2, unsigned long long* mm) {
    const Sel S = sel[blockIdx.y];
    if (S.status != 0) return;
    const Win w = win[blockIdx.y];
    double* out = vals2 + (size_t)blockIdx.y * kSel;
    unsigned long long* cw = cnt2 + blockIdx.y;
    unsigned long long* m = mm + 2 * blockIdx.y;
    const unsigned long long* cn = cand_n + (size_t)blockIdx.y * nslice;
    const long long n = w.cand_slice * nslice;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        if (!psf_cand_at(w, cn, t)) continue;
        const double v = r2[w.cand_off + t];
        if (psf_sub(v, S.a, S.s2) == S.sub) {
            const unsigned long long k = atomicAdd(cw, 1ull);
            if (k < (unsigned long long)kSel) out[k] = v;
            const unsigned long long bits = (unsigned long long)__double_as_longlong(v);  // r2 >= +0
            atomicMax(m, ~bits);
            atomicMax(m + 1, bits);
        }
    }
}

// Final selection by counting: the value v with #(< v) <= rank2 < #(<= v).
// out[4w..] = (N, cx, cy, R80); stat[w] = final status.
__global__ void psf_select(const double* res, const Sel* sel, const double* vals2, const unsigned long long* cnt2,
                           const unsigned long long* mm, double* out, int* stat) {
    __shared__ double v[kSel];
    const int w = blockIdx.x;
    const Sel S = sel[w];
    const double* R = res + kRes * w;
    const bool any = R[0] > 0.0;
    if (threadIdx.x == 0) {
        out[4 * w + 0] = R[0];
        out[4 * w + 1] = any ? R[1] : NAN;
        out[4 * w + 2] = any ? R[2] : NAN;
        out[4 * w + 3] = NAN;
        stat[w] = S.status;
    }
    if (S.status != 0) return;
    const long long c = (long long)cnt2[w];
    if (c != S.cap2 || S.rank2 < 0 || S.rank2 >= c) {
        if (threadIdx.x == 0) stat[w] = 3;
        return;
    }
    const double vmin = __longlong_as_double((long long)~mm[2 * w]), vmax = __longlong_as_double((long long)mm[2 * w + 1]);
    if (c > kSel) {
        if (threadIdx.x == 0) {
            if (vmin == vmax)
                out[4 * w + 3] = sqrt(vmin);  // all equal
            else
                stat[w] = 1;
        }
        return;
    }
    const int n = (int)c;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = vals2[(size_t)w * kSel + i];
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double x = v[i];
        int less = 0, leq = 0;
        for (int j = 0; j < n; ++j) {
            less += v[j] < x;
            leq += v[j] <= x;
        }
        if (less <= S.rank2 && S.rank2 < leq) out[4 * w + 3] = sqrt(x);  // equal values: same result
    }
}

template <typename T>
int psf_impl(robast_geom* g, const uint8_t* st, const T* fxy, long long ld, int nw, const long long* starts,
             const long long* counts, cudaStream_t s, double* result) {
    long long maxcount = 0;
    for (int w = 0; w < nw; ++w) maxcount = std::max(maxcount, counts[w]);
    const int bx = psf_blocks_per_window(nw, maxcount);
    // candidate list: per window about min(count, kCandPerWindow, kCandTotal / nw) entries, in bx
    // slices (one per block of the compaction pass)
    std::vector<Win> hw(nw);
    long long ncand = 0, maxcap = 0;
    for (int w = 0; w < nw; ++w) {
        const long long cap = std::min({counts[w], kCandPerWindow, std::max(1LL, kCandTotal / nw)});
        const long long slice = std::max(1LL, (cap + bx - 1) / bx);
        hw[w] = Win{starts[w], counts[w], ncand, slice};
        ncand += slice * bx;
        maxcap = std::max(maxcap, slice * bx);
    }
    // scratch: win | part | {res, out, stat, sel} (read back together) |
    //          {hist, hist2, cnt2, mm, cand_n} (cleared together) | vals2 | cand | cand_r2 |
    //          fallback: sel4, cnt, cap, vals
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        const size_t at = off;
        off += align16(bytes);
        return at;
    };
    const size_t o_win = carve(nw * sizeof(Win)), o_part = carve((size_t)nw * bx * 5 * 8);
    const size_t o_back = off, o_res = carve((size_t)nw * kRes * 8), o_out = carve((size_t)nw * 32),
                 o_stat = carve((size_t)nw * 4), o_sel = carve((size_t)nw * sizeof(Sel));
    const size_t back_bytes = off - o_back;
    const size_t o_zero = off, o_hist = carve((size_t)nw * (kBins + 1) * 8), o_hist2 = carve((size_t)nw * kSub * 8),
                 o_cnt2 = carve((size_t)nw * 8), o_mm = carve((size_t)nw * 16), o_candn = carve((size_t)nw * bx * 8);
    const size_t zero_bytes = off - o_zero;
    const size_t o_vals2 = carve((size_t)nw * kSel * 8);
    const size_t o_cand = carve((size_t)ncand * 8), o_r2 = carve((size_t)ncand * 8);
    const size_t o_sel4 = carve((size_t)nw * 32), o_cnt = carve((size_t)nw * 8), o_cap = carve((size_t)nw * 8);
    const size_t o_vals = off;
    std::lock_guard<std::mutex> lk(g->mu);
    int rc = grow(&g->scratch, &g->scratch_bytes, o_vals + 4096 * 8, "robast_psf");
    if (rc) return rc;
    const size_t win_bytes = align16(nw * sizeof(Win));
    rc = grow_pinned(g, win_bytes + back_bytes, "robast_psf");
    if (rc) return rc;
    unsigned char* hp = static_cast<unsigned char*>(g->pinned);  // [windows | read-back region]
    std::memcpy(hp, hw.data(), nw * sizeof(Win));
    unsigned char* b = static_cast<unsigned char*>(g->scratch);
    CU(cudaMemcpyAsync(b + o_win, hp, nw * sizeof(Win), cudaMemcpyHostToDevice, s), "robast_psf: copy");
    CU(cudaMemsetAsync(b + o_zero, 0, zero_bytes, s), "robast_psf: clear");
    const Win* dwin = reinterpret_cast<const Win*>(b + o_win);
    double* part = reinterpret_cast<double*>(b + o_part);
    double* res = reinterpret_cast<double*>(b + o_res);
    Sel* sel = reinterpret_cast<Sel*>(b + o_sel);
    auto u64 = [&](size_t o) { return reinterpret_cast<unsigned long long*>(b + o); };
    long long* cand = reinterpret_cast<long long*>(b + o_cand);
    double* cand_r2 = reinterpret_cast<double*>(b + o_r2);
    const dim3 grid(bx, nw);
    const dim3 cgrid((unsigned)std::max(1LL, std::min<long long>(std::max(1, kPartBlocks / nw), (maxcap + 1023) / 1024)), nw);
    psf_sums<T><<<grid, kRedBlock, 0, s>>>(st, fxy, ld, dwin, part);
    psf_finish<<<nw, 32, 0, s>>>(part, bx, sizeof(T) == 4 ? 1 : 0, res);
    psf_hist<T><<<grid, kRedBlock, 0, s>>>(st, fxy, ld, dwin, res, u64(o_hist));
    psf_pick1<<<nw, kScanBlock, 0, s>>>(u64(o_hist), res, dwin, bx, sel);
    psf_compact<T><<<grid, kRedBlock, 0, s>>>(st, fxy, ld, dwin, res, sel, cand, u64(o_candn));
    psf_cand_check<<<nw, 32, 0, s>>>(dwin, u64(o_candn), bx, sel);
    psf_cand_r2<T><<<cgrid, kRedBlock, 0, s>>>(fxy, ld, dwin, res, sel, cand, u64(o_candn), bx, cand_r2);
    psf_hist2<<<cgrid, kRedBlock, 0, s>>>(dwin, sel, cand_r2, u64(o_candn), bx, u64(o_hist2));
    psf_pick2<<<nw, kScanBlock, 0, s>>>(u64(o_hist2), sel);
    psf_collect2<<<cgrid, kRedBlock, 0, s>>>(dwin, sel, cand_r2, u64(o_candn), bx,
                                            reinterpret_cast<double*>(b + o_vals2), u64(o_cnt2), u64(o_mm));
    psf_select<<<nw, kScanBlock, 0, s>>>(res, sel, reinterpret_cast<const double*>(b + o_vals2), u64(o_cnt2), u64(o_mm),
                                         reinterpret_cast<double*>(b + o_out), reinterpret_cast<int*>(b + o_stat));
    CU(cudaGetLastError(), "robast_psf: launch");
    CU(cudaMemcpyAsync(hp + win_bytes, b + o_back, back_bytes, cudaMemcpyDeviceToHost, s), "robast_psf: copy");
    CU(cudaStreamSynchronize(s), "robast_psf: synchronize");
    std::vector<unsigned char> back(hp + win_bytes, hp + win_bytes + back_bytes);
    const double* hout = reinterpret_cast<const double*>(back.data() + (o_out - o_back));
    const int* hstat = reinterpret_cast<const int*>(back.data() + (o_stat - o_back));
    const Sel* hsel = reinterpret_cast<const Sel*>(back.data() + (o_sel - o_back));
    bool fallback = false;
    for (int w = 0; w < nw; ++w) {
        for (int c = 0; c < 4; ++c) result[4 * w + c] = hout[4 * w + c];
        if (hstat[w] == 3) return fail(ROBAST_E_CUDA, "robast_psf: histogram and selection disagree in window %d", w);
        fallback = fallback || hstat[w] == 1;
    }
    if (!fallback) return 0;

    // fallback for unresolved windows: collect bins lo..hi, select on the host
    std::vector<long long> sel4(4 * nw), cap(nw);
    long long total = 0;
    for (int w = 0; w < nw; ++w) {
        const bool on = hstat[w] == 1;
        sel4[4 * w] = on ? hsel[w].lo : -1;
        sel4[4 * w + 1] = on ? hsel[w].hi : -2;
        sel4[4 * w + 2] = total;
        sel4[4 * w + 3] = 0;
        cap[w] = on ? hsel[w].cap1 : 0;
        total += cap[w];
    }
    rc = grow(&g->scratch, &g->scratch_bytes, o_vals + std::max<long long>(total, 1) * 8, "robast_psf");
    if (rc) return rc;
    b = static_cast<unsigned char*>(g->scratch);  // may have moved: re-upload what the collect pass reads
    CU(cudaMemcpyAsync(b + o_win, hw.data(), nw * sizeof(Win), cudaMemcpyHostToDevice, s), "robast_psf: copy");
    CU(cudaMemcpyAsync(b + o_res, back.data() + (o_res - o_back), (size_t)nw * kRes * 8, cudaMemcpyHostToDevice, s),
       "robast_psf: copy");
    CU(cudaMemsetAsync(b + o_cnt, 0, nw * 8, s), "robast_psf: clear");
    CU(cudaMemcpyAsync(b + o_sel4, sel4.data(), nw * 32, cudaMemcpyHostToDevice, s), "robast_psf: copy");
    CU(cudaMemcpyAsync(b + o_cap, cap.data(), nw * 8, cudaMemcpyHostToDevice, s), "robast_psf: copy");
    double* vals = reinterpret_cast<double*>(b + o_vals);
    psf_collect<T><<<grid, kRedBlock, 0, s>>>(st, fxy, ld, reinterpret_cast<const Win*>(b + o_win),
                                              reinterpret_cast<const double*>(b + o_res),
                                              reinterpret_cast<const long long*>(b + o_sel4), vals, u64(o_cnt),
                                              reinterpret_cast<const long long*>(b + o_cap));
    CU(cudaGetLastError(), "robast_psf: launch");
    std::vector<double> hv(std::max<long long>(total, 1));
    std::vector<unsigned long long> got(nw);
    CU(cudaMemcpyAsync(got.data(), u64(o_cnt), nw * 8, cudaMemcpyDeviceToHost, s), "robast_psf: copy");
    if (total) CU(cudaMemcpyAsync(hv.data(), vals, total * 8, cudaMemcpyDeviceToHost, s), "robast_psf: copy");
    CU(cudaStreamSynchronize(s), "robast_psf: synchronize");
    for (int w = 0; w < nw; ++w) {
        if (hstat[w] != 1) continue;
        if ((long long)got[w] != cap[w])
            return fail(ROBAST_E_CUDA, "robast_psf: histogram and selection disagree in window %d", w);
        auto first = hv.begin() + sel4[4 * w + 2];
        std::nth_element(first, first + hsel[w].rank1, first + cap[w]);
        result[4 * w + 3] = std::sqrt(first[hsel[w].rank1]);  // the selected photon's radius
    }
    return 0;
}
}  // namespace

extern "C" int robast_psf(robast_geom* g, const uint8_t* status, const void* focal_xy, int64_t ld, int32_t n_windows,
                          const int64_t* starts, const int64_t* counts, int32_t precision, void* stream,
                          double* results) {
    if (!g || !status || !focal_xy || !results || !starts || !counts)
        return fail(ROBAST_E_NULL, "robast_psf: NULL argument");
    if (n_windows <= 0 || n_windows > 65535) return fail(ROBAST_E_INVALID, "robast_psf: n_windows must be in 1..65535");
    for (int w = 0; w < n_windows; ++w)
        if (starts[w] < 0 || counts[w] <= 0 || starts[w] + counts[w] > ld)
            return fail(ROBAST_E_INVALID, "robast_psf: window %d [%lld, +%lld) must lie inside [0, ld = %lld)", w,
                        (long long)starts[w], (long long)counts[w], (long long)ld);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long* st = reinterpret_cast<const long long*>(starts);
    const long long* ct = reinterpret_cast<const long long*>(counts);
    if (precision == 32)
        return psf_impl<float>(g, status, static_cast<const float*>(focal_xy), ld, n_windows, st, ct, s, results);
    if (precision == 64)
        return psf_impl<double>(g, status, static_cast<const double*>(focal_xy), ld, n_windows, st, ct, s, results);
    return fail(ROBAST_E_INVALID, "robast_psf: precision must be 32 or 64");
}

// ------------------------------------------------------- ALU peak probe
// Throughput of dependent-free FMA chains (8 independent accumulators per
// thread), all SMs busy: the denominator of the ALU roofline.
namespace {
template <typename T>
__global__ void fma_probe(T* sink, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = x[k] * a + b;
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == (T)1234.5678) sink[0] = s;  // keeps the chains alive
}
}  // namespace

extern "C" int robast_measure_alu_peak(int32_t precision, void* stream, double* flops_per_s) {
    if (!flops_per_s) return fail(ROBAST_E_NULL, "robast_measure_alu_peak: result pointer is NULL");
    if (precision != 32 && precision != 64) return fail(ROBAST_E_INVALID, "robast_measure_alu_peak: precision 32 or 64");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    CU(cudaGetDevice(&dev), "robast_measure_alu_peak");
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "robast_measure_alu_peak");
    void* sink = nullptr;
    CU(cudaMalloc(&sink, 64), "robast_measure_alu_peak: cudaMalloc");
    const int block = 256, grid = sms * 8;
    const int iters = precision == 32 ? 1 << 14 : 1 << 9;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 6; ++rep) {
        cudaEventRecord(e0, s);
        if (precision == 32)
            fma_probe<float><<<grid, block, 0, s>>>((float*)sink, iters, 0.999999f, 1e-7f);
        else
            fma_probe<double><<<grid, block, 0, s>>>((double*)sink, iters, 0.999999, 1e-7);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;  // first launch is warm-up
    }
    cudaError_t e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) return cuda_fail(e, "robast_measure_alu_peak");
    *flops_per_s = 2.0 * 8.0 * (double)iters * (double)block * (double)grid / (best * 1e-3);
    return 0;
}

// ============================================ allocation-free spot diagram
// robast_psf_noalloc: the spot-diagram statistics of robast_psf computed
// without allocating anything.
//
// Some callers cannot allocate device memory at the time they want these
// statistics: code under a caching allocator that owns all device memory, or
// embedders whose memory budget is fixed up front.  This entry point serves
// them.  It synchronises the caller's stream between its histogram rounds and
// reads their results on the host, so it must not be issued on a stream that
// is being captured into a CUDA graph.  Its
// scratch lives in one file-scope __device__ array of fixed size (about
// 6.4 MB) that every GPU which loads the library holds until the process
// exits; it calls no cudaMalloc, cudaFree or allocating library routine, and
// its host-side buffers are static too.
//
// Limits: at most NA_MAX_WINDOWS windows per call.  Because the scratch is
// bounded, the selection of the 80% radius does not collect a whole
// histogram bin (which can hold any number of photons): it refines the bin
// that holds the rank with further 4096-bin histograms until that bin holds
// at most NA_CAP values, then selects among them exactly; a bin still over
// NA_CAP after NA_ROUNDS rounds spans only a few doubles, whose copies are
// counted one value at a time.  The result is the same number robast_psf
// returns.
//
// Sharing: every call on a device uses the same scratch array and leaves its
// contents behind; each call clears what must start at zero.  Calls whose GPU
// work overlaps (several host threads, or several streams) race on it; the
// host-side part is serialised by a mutex, but work already queued on one
// stream is not ordered against another stream's.
//
// Set-up: the first call on a device looks up the array's device address with
// cudaGetSymbolAddress (with that device current) and caches it; make that
// first call before any stream capture begins on the device.
namespace {

constexpr int NA_MAX_WINDOWS = 64;
constexpr int NA_BINS = 4096;  // + 1 overflow bin in the first round
constexpr int NA_CAP = 8192;   // values collected per window for the final selection
constexpr int NA_ROUNDS = 8;   // histogram rounds (4096^8 resolves any double interval)
constexpr int NA_BLOCK = 256;
constexpr int NA_MAX_PART_BLOCKS = kPartBlocks;
constexpr int NA_MAX_DEVICES = 64;

struct NaScratch {
    double part[NA_MAX_PART_BLOCKS * 5];
    double res[NA_MAX_WINDOWS * 4];  // N, cx, cy, first-round range
    int chosen[NA_MAX_WINDOWS * NA_ROUNDS];
    double lohi[NA_MAX_WINDOWS * NA_ROUNDS * 2];
    unsigned long long hist[NA_MAX_WINDOWS * (NA_BINS + 1)];
    unsigned long long cnt[NA_MAX_WINDOWS];
    unsigned long long rmax_bits[NA_MAX_WINDOWS];
    unsigned long long rmin_bits[NA_MAX_WINDOWS];
    double vals[NA_MAX_WINDOWS * NA_CAP];
};

// The scratch: one per device, shared by every call (see the header comment).
static __device__ __align__(256) NaScratch g_na_scratch;

struct WinSet {
    int n;
    int round;  // histogram round of this launch
    long long start[NA_MAX_WINDOWS];
    long long count[NA_MAX_WINDOWS];
};

template <typename T>
__global__ void na_sums(const uint8_t* st, const T* fxy, long long ld, WinSet ws, NaScratch* S) {
    const int w = blockIdx.y;
    double acc[5];
    psf_thread_sums(st, fxy, ld, ws.start[w], ws.count[w], blockIdx.x * (long long)blockDim.x + threadIdx.x,
                    (long long)gridDim.x * blockDim.x, acc);
    __shared__ double sh[5][NA_BLOCK];
    for (int c = 0; c < 5; ++c) sh[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int h = NA_BLOCK / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int c = 0; c < 5; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 5; ++c) S->part[((size_t)w * gridDim.x + blockIdx.x) * 5 + c] = sh[c][0];
}

// one warp per window, the same fixed-order sums as robast_psf
__global__ void na_finish(int nblocks, NaScratch* S) {
    const int w = blockIdx.x;
    double a[5];
    psf_window_sums(S->part, nblocks, w, a);
    if (threadIdx.x != 0) return;
    const double n = a[0];
    const double cx = n > 0 ? a[1] / n : 0.0, cy = n > 0 ? a[2] / n : 0.0;
    const double ms = n > 0 ? fmax(0.0, (a[3] + a[4]) / n - cx * cx - cy * cy) : 0.0;
    S->res[4 * w + 0] = n;
    S->res[4 * w + 1] = cx;
    S->res[4 * w + 2] = cy;
    S->res[4 * w + 3] = fmax(8.0 * sqrt(ms), 1e-300);
}

// bin of r in round j of window w: round 0 covers [0, range) plus an overflow
// bin; later rounds cover [lo, hi) of the bin chosen before (clamped)
__device__ __forceinline__ int na_bin(const NaScratch* S, int w, int j, double r) {
    if (j == 0) {
        const double range = S->res[4 * w + 3];
        if (!(r < range)) return NA_BINS;
        int b = (int)(r / range * NA_BINS);
        return b < 0 ? 0 : (b >= NA_BINS ? NA_BINS - 1 : b);
    }
    const double lo = S->lohi[(w * NA_ROUNDS + j) * 2], hi = S->lohi[(w * NA_ROUNDS + j) * 2 + 1];
    int b = hi > lo ? (int)((r - lo) / (hi - lo) * NA_BINS) : 0;
    return b < 0 ? 0 : (b >= NA_BINS ? NA_BINS - 1 : b);
}

template <typename T>
__device__ __forceinline__ bool na_member(const uint8_t* st, const T* fxy, long long ld, long long i, int w, int upto,
                                          const NaScratch* S, double* r) {
    if (st[i] != ROBAST_ST_DETECTED) return false;
    const double dx = (double)fxy[i] - S->res[4 * w + 1], dy = (double)fxy[ld + i] - S->res[4 * w + 2];
    *r = sqrt(dx * dx + dy * dy);
    for (int j = 0; j < upto; ++j)
        if (na_bin(S, w, j, *r) != S->chosen[w * NA_ROUNDS + j]) return false;
    return true;
}

// histogram of round ws.round over the values that followed every earlier choice
template <typename T>
__global__ void na_hist(const uint8_t* st, const T* fxy, long long ld, WinSet ws, NaScratch* S) {
    __shared__ unsigned int h[NA_BINS + 1];
    for (int k = threadIdx.x; k <= NA_BINS; k += blockDim.x) h[k] = 0;
    __syncthreads();
    const int w = blockIdx.y;
    if (S->chosen[w * NA_ROUNDS + ws.round] == -2) {  // -2 marks a window still refining
        for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < ws.count[w];
             k += (long long)gridDim.x * blockDim.x) {
            double r;
            if (na_member(st, fxy, ld, ws.start[w] + k, w, ws.round, S, &r))
                atomicAdd(&h[na_bin(S, w, ws.round, r)], 1u);
        }
    }
    __syncthreads();
    unsigned long long* H = S->hist + (size_t)w * (NA_BINS + 1);
    for (int k = threadIdx.x; k <= NA_BINS; k += blockDim.x)
        if (h[k]) atomicAdd(H + k, (unsigned long long)h[k]);
}

// largest radius among the values of the first-round overflow bin
template <typename T>
__global__ void na_rmax(const uint8_t* st, const T* fxy, long long ld, WinSet ws, NaScratch* S) {
    const int w = blockIdx.y;
    double m = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < ws.count[w];
         k += (long long)gridDim.x * blockDim.x) {
        double r;
        if (na_member(st, fxy, ld, ws.start[w] + k, w, 1, S, &r)) m = fmax(m, r);
    }
    unsigned long long bits = (unsigned long long)__double_as_longlong(m);
    for (int off = 16; off > 0; off >>= 1) bits = max(bits, __shfl_xor_sync(0xffffffffu, bits, off));
    if ((threadIdx.x & 31) == 0) atomicMax(S->rmax_bits + w, bits);
}

// values of the final bin (chosen in rounds 0 .. ws.round - 1), at most NA_CAP per window
template <typename T>
__global__ void na_collect(const uint8_t* st, const T* fxy, long long ld, WinSet ws, NaScratch* S, const int* upto) {
    const int w = blockIdx.y;
    const int u = upto[w];
    if (u <= 0) return;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < ws.count[w];
         k += (long long)gridDim.x * blockDim.x) {
        double r;
        if (na_member(st, fxy, ld, ws.start[w] + k, w, u, S, &r)) {
            const unsigned long long j = atomicAdd(S->cnt + w, 1ull);
            if (j < (unsigned long long)NA_CAP) S->vals[(size_t)w * NA_CAP + j] = r;
        }
    }
}

// Smallest and largest value (as bit patterns: radii are >= 0, so their bits order like the
// values) of the final bin of each window with upto[w] > 0.
template <typename T>
__global__ void na_minmax(const uint8_t* st, const T* fxy, long long ld, WinSet ws, NaScratch* S, const int* upto) {
    const int w = blockIdx.y;
    const int u = upto[w];
    if (u <= 0) return;
    unsigned long long lo = ~0ull, hi = 0ull;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < ws.count[w];
         k += (long long)gridDim.x * blockDim.x) {
        double r;
        if (na_member(st, fxy, ld, ws.start[w] + k, w, u, S, &r)) {
            const unsigned long long b = (unsigned long long)__double_as_longlong(r);
            lo = min(lo, b);
            hi = max(hi, b);
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, off));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, off));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(S->rmin_bits + w, lo);
        atomicMax(S->rmax_bits + w, hi);
    }
}

// One bin per representable double from the final bin's smallest value: counts of each
// distinct value of the final bin (its values span fewer than NA_BINS doubles).
template <typename T>
__global__ void na_ulp_hist(const uint8_t* st, const T* fxy, long long ld, WinSet ws, NaScratch* S, const int* upto) {
    const int w = blockIdx.y;
    const int u = upto[w];
    if (u <= 0) return;
    const unsigned long long b0 = S->rmin_bits[w];
    unsigned long long* H = S->hist + (size_t)w * (NA_BINS + 1);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < ws.count[w];
         k += (long long)gridDim.x * blockDim.x) {
        double r;
        if (na_member(st, fxy, ld, ws.start[w] + k, w, u, S, &r)) {
            const unsigned long long j = (unsigned long long)__double_as_longlong(r) - b0;
            if (j < (unsigned long long)NA_BINS) atomicAdd(H + j, 1ull);
        }
    }
}

// device address of the scratch, looked up once per device
std::mutex na_mu;
NaScratch* na_dev[NA_MAX_DEVICES] = {nullptr};
// static host mirrors (no allocation per call)
unsigned long long na_h_hist[NA_MAX_WINDOWS * (NA_BINS + 1)];
double na_h_vals[NA_MAX_WINDOWS * NA_CAP];
double na_h_res[NA_MAX_WINDOWS * 4];
int na_h_chosen[NA_MAX_WINDOWS * NA_ROUNDS];
double na_h_lohi[NA_MAX_WINDOWS * NA_ROUNDS * 2];
int na_h_upto[NA_MAX_WINDOWS];
unsigned long long na_h_cnt[NA_MAX_WINDOWS];
unsigned long long na_h_rmax[NA_MAX_WINDOWS];
unsigned long long na_h_rmin[NA_MAX_WINDOWS];
int na_h_over[NA_MAX_WINDOWS];

template <typename T>
int na_impl(NaScratch* S, const uint8_t* st, const T* fxy, long long ld, const WinSet& ws0, cudaStream_t s,
            double* results) {
    WinSet ws = ws0;
    const int nw = ws.n;
    long long maxcount = 0;
    for (int w = 0; w < nw; ++w) maxcount = std::max(maxcount, ws.count[w]);
    // same block partition of the sums as robast_psf, so the centroids agree bit for bit
    const int bx = psf_blocks_per_window(nw, maxcount);
    const dim3 grid(bx, nw);
    na_sums<T><<<grid, NA_BLOCK, 0, s>>>(st, fxy, ld, ws, S);
    na_finish<<<nw, 32, 0, s>>>(bx, S);
    CU(cudaGetLastError(), "robast_psf_noalloc: launch");
    CU(cudaMemcpyAsync(na_h_res, S->res, nw * 4 * sizeof(double), cudaMemcpyDeviceToHost, s),
          "robast_psf_noalloc: copy");
    CU(cudaStreamSynchronize(s), "robast_psf_noalloc: synchronize");
    long long rank[NA_MAX_WINDOWS];
    bool active[NA_MAX_WINDOWS];
    for (int w = 0; w < nw; ++w) {
        const long long N = (long long)na_h_res[4 * w];
        results[4 * w + 0] = na_h_res[4 * w];
        results[4 * w + 1] = N ? na_h_res[4 * w + 1] : NAN;
        results[4 * w + 2] = N ? na_h_res[4 * w + 2] : NAN;
        results[4 * w + 3] = NAN;
        rank[w] = N ? (long long)std::ceil(0.8 * (double)N) - 1 : -1;
        active[w] = N > 0;
        na_h_upto[w] = 0;
        for (int j = 0; j < NA_ROUNDS; ++j) na_h_chosen[w * NA_ROUNDS + j] = active[w] ? -2 : -1;
    }
    int round = 0;
    bool any = true;
    while (any) {
        CU(cudaMemcpyAsync(S->chosen, na_h_chosen, sizeof(int) * nw * NA_ROUNDS, cudaMemcpyHostToDevice, s),
              "robast_psf_noalloc: copy");
        CU(cudaMemcpyAsync(S->lohi, na_h_lohi, sizeof(double) * nw * NA_ROUNDS * 2, cudaMemcpyHostToDevice, s),
              "robast_psf_noalloc: copy");
        CU(cudaMemsetAsync(S->hist, 0, sizeof(unsigned long long) * nw * (NA_BINS + 1), s),
              "robast_psf_noalloc: clear");
        ws.round = round;
        na_hist<T><<<grid, NA_BLOCK, 0, s>>>(st, fxy, ld, ws, S);
        CU(cudaGetLastError(), "robast_psf_noalloc: launch");
        CU(cudaMemcpyAsync(na_h_hist, S->hist, sizeof(unsigned long long) * nw * (NA_BINS + 1),
                              cudaMemcpyDeviceToHost, s),
              "robast_psf_noalloc: copy");
        CU(cudaStreamSynchronize(s), "robast_psf_noalloc: synchronize");
        bool need_rmax = false;
        any = false;
        for (int w = 0; w < nw; ++w) {
            if (!active[w]) continue;
            const unsigned long long* H = na_h_hist + (size_t)w * (NA_BINS + 1);
            long long acc = 0;
            int b = 0;
            for (; b <= NA_BINS; ++b) {
                if (acc + (long long)H[b] > rank[w]) break;
                acc += (long long)H[b];
            }
            if (b > NA_BINS) return fail(ROBAST_E_CUDA, "robast_psf_noalloc: rank not found in window %d", w);
            rank[w] -= acc;
            na_h_chosen[w * NA_ROUNDS + round] = b;
            const long long inbin = (long long)H[b];
            const bool last_round = round + 1 >= NA_ROUNDS;
            if (inbin <= NA_CAP || last_round) {
                active[w] = false;
                na_h_upto[w] = round + 1;
                for (int j = round + 1; j < NA_ROUNDS; ++j) na_h_chosen[w * NA_ROUNDS + j] = -1;
                continue;
            }
            // refine this bin in the next round
            double lo, hi;
            if (round == 0) {
                const double range = na_h_res[4 * w + 3];
                if (b == NA_BINS) {
                    need_rmax = true;  // interval [range, max r] fixed after the max pass
                    lo = range;
                    hi = range;
                } else {
                    lo = range * b / NA_BINS;
                    hi = range * (b + 1) / NA_BINS;
                }
            } else {
                const double plo = na_h_lohi[(w * NA_ROUNDS + round) * 2];
                const double phi = na_h_lohi[(w * NA_ROUNDS + round) * 2 + 1];
                lo = plo + (phi - plo) * b / NA_BINS;
                hi = plo + (phi - plo) * (b + 1) / NA_BINS;
            }
            // the next round's bins span a little beyond the computed edges: membership is
            // decided by the chain of bin indices, the interval only spreads the values
            const double pad = (hi - lo) * 1e-9 + 4.0 * std::fabs(hi) * 2.220446049250313e-16;
            na_h_lohi[(w * NA_ROUNDS + round + 1) * 2] = lo - pad;
            na_h_lohi[(w * NA_ROUNDS + round + 1) * 2 + 1] = hi + pad;
            na_h_chosen[w * NA_ROUNDS + round + 1] = -2;
            any = true;
        }
        if (need_rmax) {
            CU(cudaMemcpyAsync(S->chosen, na_h_chosen, sizeof(int) * nw * NA_ROUNDS, cudaMemcpyHostToDevice, s),
                  "robast_psf_noalloc: copy");
            CU(cudaMemsetAsync(S->rmax_bits, 0, sizeof(unsigned long long) * nw, s), "robast_psf_noalloc: clear");
            na_rmax<T><<<grid, NA_BLOCK, 0, s>>>(st, fxy, ld, ws, S);
            CU(cudaGetLastError(), "robast_psf_noalloc: launch");
            CU(cudaMemcpyAsync(na_h_rmax, S->rmax_bits, sizeof(unsigned long long) * nw, cudaMemcpyDeviceToHost, s),
                  "robast_psf_noalloc: copy");
            CU(cudaStreamSynchronize(s), "robast_psf_noalloc: synchronize");
            for (int w = 0; w < nw; ++w) {
                if (!active[w] || round != 0 || na_h_chosen[w * NA_ROUNDS] != NA_BINS) continue;
                double rmax;
                std::memcpy(&rmax, &na_h_rmax[w], sizeof rmax);
                na_h_lohi[(w * NA_ROUNDS + 1) * 2 + 1] = rmax * (1.0 + 1e-12) + 1e-300;
            }
        }
        ++round;
    }
    // collect the final bins and select
    CU(cudaMemcpyAsync(S->chosen, na_h_chosen, sizeof(int) * nw * NA_ROUNDS, cudaMemcpyHostToDevice, s),
          "robast_psf_noalloc: copy");
    CU(cudaMemcpyAsync(S->lohi, na_h_lohi, sizeof(double) * nw * NA_ROUNDS * 2, cudaMemcpyHostToDevice, s),
          "robast_psf_noalloc: copy");
    CU(cudaMemsetAsync(S->cnt, 0, sizeof(unsigned long long) * nw, s), "robast_psf_noalloc: clear");
    // the per-window round counts travel in the part[] area, unused from here on
    CU(cudaMemcpyAsync(S->part, na_h_upto, sizeof(int) * nw, cudaMemcpyHostToDevice, s), "robast_psf_noalloc: copy");
    na_collect<T><<<grid, NA_BLOCK, 0, s>>>(st, fxy, ld, ws, S, reinterpret_cast<const int*>(S->part));
    CU(cudaGetLastError(), "robast_psf_noalloc: launch");
    CU(cudaMemcpyAsync(na_h_cnt, S->cnt, sizeof(unsigned long long) * nw, cudaMemcpyDeviceToHost, s),
          "robast_psf_noalloc: copy");
    CU(cudaMemcpyAsync(na_h_vals, S->vals, sizeof(double) * (size_t)nw * NA_CAP, cudaMemcpyDeviceToHost, s),
          "robast_psf_noalloc: copy");
    CU(cudaStreamSynchronize(s), "robast_psf_noalloc: synchronize");
    bool any_over = false;
    for (int w = 0; w < nw; ++w) {
        na_h_over[w] = 0;
        if (na_h_upto[w] <= 0) continue;
        if (na_h_cnt[w] > (unsigned long long)NA_CAP) {
            // still over the cap after the last round: resolved exactly below
            na_h_over[w] = na_h_upto[w];
            any_over = true;
            continue;
        }
        const long long got = (long long)na_h_cnt[w];
        if (got <= rank[w]) return fail(ROBAST_E_CUDA, "robast_psf_noalloc: selection lost values in window %d", w);
        double* v = na_h_vals + (size_t)w * NA_CAP;
        std::nth_element(v, v + rank[w], v + got);
        results[4 * w + 3] = v[rank[w]];
    }
    if (any_over) {
        // A final bin over the cap is a few ulps wide (each round pads its interval by 4 ulps
        // of its upper edge), so it holds a few distinct doubles with many copies each: count
        // the copies of every distinct value and take the rank's, the same exact nearest-rank
        // value that robast_psf selects, whatever the order of the atomics.
        CU(cudaMemcpyAsync(S->part, na_h_over, sizeof(int) * nw, cudaMemcpyHostToDevice, s), "robast_psf_noalloc: copy");
        CU(cudaMemsetAsync(S->rmin_bits, 0xff, sizeof(unsigned long long) * nw, s), "robast_psf_noalloc: clear");
        CU(cudaMemsetAsync(S->rmax_bits, 0, sizeof(unsigned long long) * nw, s), "robast_psf_noalloc: clear");
        na_minmax<T><<<grid, NA_BLOCK, 0, s>>>(st, fxy, ld, ws, S, reinterpret_cast<const int*>(S->part));
        CU(cudaGetLastError(), "robast_psf_noalloc: launch");
        CU(cudaMemcpyAsync(na_h_rmin, S->rmin_bits, sizeof(unsigned long long) * nw, cudaMemcpyDeviceToHost, s),
           "robast_psf_noalloc: copy");
        CU(cudaMemcpyAsync(na_h_rmax, S->rmax_bits, sizeof(unsigned long long) * nw, cudaMemcpyDeviceToHost, s),
           "robast_psf_noalloc: copy");
        CU(cudaStreamSynchronize(s), "robast_psf_noalloc: synchronize");
        for (int w = 0; w < nw; ++w)
            if (na_h_over[w] && na_h_rmax[w] - na_h_rmin[w] >= (unsigned long long)NA_BINS)
                return fail(ROBAST_E_INVALID,
                            "robast_psf_noalloc: window %d: the rank's bin still spans %llu doubles after %d rounds", w,
                            na_h_rmax[w] - na_h_rmin[w] + 1, NA_ROUNDS);
        CU(cudaMemsetAsync(S->hist, 0, sizeof(unsigned long long) * nw * (NA_BINS + 1), s), "robast_psf_noalloc: clear");
        na_ulp_hist<T><<<grid, NA_BLOCK, 0, s>>>(st, fxy, ld, ws, S, reinterpret_cast<const int*>(S->part));
        CU(cudaGetLastError(), "robast_psf_noalloc: launch");
        CU(cudaMemcpyAsync(na_h_hist, S->hist, sizeof(unsigned long long) * nw * (NA_BINS + 1), cudaMemcpyDeviceToHost, s),
           "robast_psf_noalloc: copy");
        CU(cudaStreamSynchronize(s), "robast_psf_noalloc: synchronize");
        for (int w = 0; w < nw; ++w) {
            if (!na_h_over[w]) continue;
            const unsigned long long* H = na_h_hist + (size_t)w * (NA_BINS + 1);
            long long acc = 0;
            int b = 0;
            for (; b < NA_BINS; ++b) {
                if (acc + (long long)H[b] > rank[w]) break;
                acc += (long long)H[b];
            }
            if (b >= NA_BINS) return fail(ROBAST_E_CUDA, "robast_psf_noalloc: rank not found in window %d", w);
            const unsigned long long bits = na_h_rmin[w] + (unsigned long long)b;
            double v;
            std::memcpy(&v, &bits, sizeof v);
            results[4 * w + 3] = v;
        }
    }
    return 0;
}

}  // namespace

extern "C" int robast_psf_noalloc(const uint8_t* status, const void* focal_xy, int64_t ld, int32_t n_windows,
                                  const int64_t* starts, const int64_t* counts, int32_t precision, void* stream,
                                  double* results) {
    if (!status || !focal_xy || !results || !starts || !counts)
        return fail(ROBAST_E_NULL, "robast_psf_noalloc: NULL argument");
    if (n_windows <= 0 || n_windows > NA_MAX_WINDOWS)
        return fail(ROBAST_E_INVALID, "robast_psf_noalloc: n_windows must be in 1..%d (got %d)", NA_MAX_WINDOWS,
                       n_windows);
    if (precision != 32 && precision != 64)
        return fail(ROBAST_E_INVALID, "robast_psf_noalloc: precision must be 32 or 64");
    WinSet ws{};
    ws.n = n_windows;
    for (int w = 0; w < n_windows; ++w) {
        if (starts[w] < 0 || counts[w] <= 0 || starts[w] + counts[w] > ld)
            return fail(ROBAST_E_INVALID, "robast_psf_noalloc: window %d [%lld, +%lld) must lie inside [0, ld = %lld)",
                           w, (long long)starts[w], (long long)counts[w], (long long)ld);
        ws.start[w] = starts[w];
        ws.count[w] = counts[w];
    }
    std::lock_guard<std::mutex> lk(na_mu);
    int dev = 0;
    CU(cudaGetDevice(&dev), "robast_psf_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= NA_MAX_DEVICES) return fail(ROBAST_E_UNSUPPORTED, "robast_psf_noalloc: device %d", dev);
    if (!na_dev[dev]) {
        // the array's name is only a host-side stand-in: fetch its device address once
        void* p = nullptr;
        CU(cudaGetSymbolAddress(&p, g_na_scratch), "robast_psf_noalloc: cudaGetSymbolAddress");
        na_dev[dev] = static_cast<NaScratch*>(p);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == 32)
        return na_impl<float>(na_dev[dev], status, static_cast<const float*>(focal_xy), ld, ws, s, results);
    return na_impl<double>(na_dev[dev], status, static_cast<const double*>(focal_xy), ld, ws, s, results);
}
