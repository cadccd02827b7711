/*
 * FP64 CPU oracle for the non-sequential photon trace -- TEST INFRASTRUCTURE.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg load
 * this library.  The GPU path shares no code with it.
 *
 * It is deliberately plain: brute-force nearest hit over every surface of the
 * photon's optical system (no acceleration structure), scalar double
 * arithmetic, compiled with -ffp-contract=off.  Citations are to Okumura,
 * Noda, Rulten, "ROBAST: Development of a Non-Sequential Ray-Tracing
 * Simulation Library and its Applications in the Cherenkov Telescope Array",
 * ICRC 2015 (arXiv:1508.07803):
 *   Sec. 1   -- non-sequential tracing: the next surface is the nearest one
 *               hit, no surface order is given in advance.
 *   Sec. 2.1 -- the navigation supplies the hit point, the direction and the
 *               surface normal; mirrors reflect, lenses refract, the focal
 *               surface detects, obscurations absorb.
 *   Sec. 2.2 -- shapes: primitive shapes, the aspheric disk, the polygonal
 *               Winston cone and the Bezier-profile polygonal cone.
 *   Sec. 3   -- the workloads: segmented parabolic dish with masts,
 *               Schwarzschild-Couder aspheric two-mirror optics, hexagonal
 *               light concentrators.
 * The paper gives no numbers for any of the quantitative choices below; each
 * is a reading recorded in the design notes (epsilon, ties, reflectivity
 * draw, roughness, Fresnel, Newton, random streams).
 */
#include "oracle.h"

#include <cmath>
#include <algorithm>
#include <cstring>
#include <thread>
#include <vector>

namespace {

struct V3 {
    double x, y, z;
};
V3 v3(double x, double y, double z) { return V3{x, y, z}; }
V3 operator+(V3 a, V3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
V3 operator-(V3 a, V3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
V3 operator*(double s, V3 a) { return v3(s * a.x, s * a.y, s * a.z); }
double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
V3 normalize(V3 a) { return (1.0 / std::sqrt(dot(a, a))) * a; }

/* ---------------------------------------------------------------- Philox */
/* Philox4x32-10, Salmon et al. SC'11: ten rounds of two 32x32->64 multiplies
 * with a Weyl-sequence key schedule. */
void philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* uniform in (0,1) from one 32-bit word: (w + 1/2) 2^-32 */
double unit_open(uint32_t w) { return ((double)w + 0.5) * (1.0 / 4294967296.0); }

/* ------------------------------------------------------------- Surfaces */
struct Frame {
    double r[9]; /* rows: local axes in world coordinates (after tilt) */
    V3 o;
};

void mat_mul(const double a[9], const double b[9], double c[9]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += a[3 * i + k] * b[3 * k + j];
            c[3 * i + j] = s;
        }
}

/* The tilted frame: the local->world matrix M (columns = local axes) becomes
 * M Rx(alpha) Ry(beta), i.e. rotation about the local x axis by alpha, then
 * about the rotated local y axis by beta, both through the local origin.  The
 * row matrix is its transpose: Ry(beta)^T Rx(alpha)^T R. */
Frame make_frame(const o_surface& s) {
    Frame f;
    f.o = v3(s.origin[0], s.origin[1], s.origin[2]);
    double ca = std::cos(s.tilt[0]), sa = std::sin(s.tilt[0]);
    double cb = std::cos(s.tilt[1]), sb = std::sin(s.tilt[1]);
    double rxT[9] = {1, 0, 0, 0, ca, sa, 0, -sa, ca};
    double ryT[9] = {cb, 0, -sb, 0, 1, 0, sb, 0, cb};
    double tmp[9];
    mat_mul(rxT, s.rot, tmp);
    mat_mul(ryT, tmp, f.r);
    return f;
}

V3 to_local_pt(const Frame& f, V3 p) {
    V3 q = p - f.o;
    return v3(f.r[0] * q.x + f.r[1] * q.y + f.r[2] * q.z, f.r[3] * q.x + f.r[4] * q.y + f.r[5] * q.z,
              f.r[6] * q.x + f.r[7] * q.y + f.r[8] * q.z);
}
V3 to_local_vec(const Frame& f, V3 q) {
    return v3(f.r[0] * q.x + f.r[1] * q.y + f.r[2] * q.z, f.r[3] * q.x + f.r[4] * q.y + f.r[5] * q.z,
              f.r[6] * q.x + f.r[7] * q.y + f.r[8] * q.z);
}
V3 to_world_vec(const Frame& f, V3 q) {
    return v3(f.r[0] * q.x + f.r[3] * q.y + f.r[6] * q.z, f.r[1] * q.x + f.r[4] * q.y + f.r[7] * q.z,
              f.r[2] * q.x + f.r[5] * q.y + f.r[8] * q.z);
}

/* Aperture test on the local (x, y) of a hit.  Inclusive on the boundary
 * (a point on a shared facet edge belongs to every facet it touches).  The
 * returned margin is the signed distance to the nearest edge relative to the
 * aperture size: >= 0 inside. */
bool aperture_inside(const o_surface& s, double x, double y, double* margin) {
    double r2 = x * x + y * y;
    switch (s.aperture) {
        case O_AP_NONE:
            *margin = 1.0;
            return true;
        case O_AP_CIRCLE: {
            double r = std::sqrt(r2);
            *margin = (s.ap[0] - r) / s.ap[0];
            return r2 <= s.ap[0] * s.ap[0];
        }
        case O_AP_ANNULUS: {
            double r = std::sqrt(r2);
            *margin = std::fmin(r - s.ap[0], s.ap[1] - r) / s.ap[1];
            return r2 >= s.ap[0] * s.ap[0] && r2 <= s.ap[1] * s.ap[1];
        }
        case O_AP_SECTOR: {
            /* rmin <= r <= rmax and phi0 <= phi <= phi1 (span <= pi), the angle
             * test through the signs of two cross products. */
            double r = std::sqrt(r2);
            double e0x = std::cos(s.ap[2]), e0y = std::sin(s.ap[2]);
            double e1x = std::cos(s.ap[3]), e1y = std::sin(s.ap[3]);
            double c0 = e0x * y - e0y * x;  /* >= 0: counter-clockwise of edge 0 */
            double c1 = x * e1y - y * e1x;  /* >= 0: clockwise of edge 1 */
            double m = std::fmin(std::fmin(r - s.ap[0], s.ap[1] - r), std::fmin(c0, c1));
            *margin = m / s.ap[1];
            return r2 >= s.ap[0] * s.ap[0] && r2 <= s.ap[1] * s.ap[1] && c0 >= 0.0 && c1 >= 0.0;
        }
        case O_AP_HEXAGON: {
            /* flats facing 0, 60, 120 (and opposite) degrees */
            const double c60 = 0.5, s60 = std::sqrt(3.0) / 2.0;
            double a = std::fabs(x);
            double b = std::fabs(c60 * x + s60 * y);
            double c = std::fabs(-c60 * x + s60 * y);
            double m = std::fmax(a, std::fmax(b, c));
            *margin = (s.ap[0] - m) / s.ap[0];
            return m <= s.ap[0];
        }
        case O_AP_RECT: {
            double mx = s.ap[0] - std::fabs(x), my = s.ap[1] - std::fabs(y);
            *margin = std::fmin(mx / s.ap[0], my / s.ap[1]);
            return std::fabs(x) <= s.ap[0] && std::fabs(y) <= s.ap[1];
        }
    }
    *margin = -1.0;
    return false;
}

/* Radius of the circle that bounds the aperture in the local (x, y) plane. */
double aperture_bound(const o_surface& s) {
    switch (s.aperture) {
        case O_AP_CIRCLE: return s.ap[0];
        case O_AP_ANNULUS:
        case O_AP_SECTOR: return s.ap[1];
        case O_AP_HEXAGON: return s.ap[0] * 2.0 / std::sqrt(3.0);
        case O_AP_RECT: return std::sqrt(s.ap[0] * s.ap[0] + s.ap[1] * s.ap[1]);
    }
    return INFINITY;
}

bool has_asphere(const o_surface& s) {
    for (int i = 0; i < 8; ++i)
        if (s.asph[i] != 0.0) return true;
    return false;
}

/* Even-asphere sag z(rho), rho = x^2 + y^2 (Sec. 2.2, AGeoAsphericDisk):
 *   z = c rho / (1 + sqrt(1 - (1+k) c^2 rho)) + sum_i A_i rho^i, i = 1..8.
 * dz/drho = c / (2 sqrt(1 - (1+k) c^2 rho)) + sum_i i A_i rho^(i-1). */
bool sag_and_slope(const o_surface& s, double rho, double* z, double* dzdrho) {
    double c = s.curv, k = s.conic;
    double arg = 1.0 - (1.0 + k) * c * c * rho;
    if (arg < 0.0) return false;
    double sq = std::sqrt(arg);
    double zz = c * rho / (1.0 + sq);
    double slope = c / (2.0 * sq);
    double rp = rho; /* rho^i */
    double rpm = 1.0; /* rho^(i-1) */
    for (int i = 1; i <= 8; ++i) {
        zz += s.asph[i - 1] * rp;
        slope += (double)i * s.asph[i - 1] * rpm;
        rpm = rp;
        rp *= rho;
    }
    *z = zz;
    *dzdrho = slope;
    return true;
}

struct Cand {
    double t;
    double margin; /* |relative margin| */
};

struct LocalHit {
    double t;
    V3 pl;      /* local hit point */
    V3 nl;      /* local front normal (unit) */
    bool error; /* Newton failed */
};

/* Ray vs sag surface in its local frame.  The surface is the quadric
 *   F = c (x^2 + y^2 + (1+k) z^2) - 2 z = 0
 * restricted to the sag branch (1+k) c z <= 1, optionally perturbed by the
 * aspheric polynomial.  Pure conics: both roots of the quadratic in t,
 * smallest valid one.  Aspheres: Newton on f(t) = z(t) - sag(rho(t)) from the
 * first on-branch conic root, |dt| < tol, at most 32 iterations, else error. */
bool hit_sag(const o_surface& s, V3 p, V3 d, double eps, double newton_tol, LocalHit* h,
             std::vector<Cand>* cands) {
    double c = s.curv, k1 = 1.0 + s.conic;
    double a = c * (d.x * d.x + d.y * d.y + k1 * d.z * d.z);
    double b = c * (p.x * d.x + p.y * d.y + k1 * p.z * d.z) - d.z;
    double g = c * (p.x * p.x + p.y * p.y + k1 * p.z * p.z) - 2.0 * p.z;
    double roots[2];
    int nr = 0;
    if (a == 0.0) {
        if (b != 0.0) roots[nr++] = -g / (2.0 * b);
    } else {
        double disc = b * b - a * g;
        if (disc >= 0.0) {
            double sq = std::sqrt(disc);
            double q = -(b + (b >= 0.0 ? sq : -sq));
            if (q != 0.0) {
                double t1 = q / a, t2 = g / q;
                roots[nr++] = std::fmin(t1, t2);
                roots[nr++] = std::fmax(t1, t2);
            } else {
                roots[nr++] = 0.0; /* b = 0 and g = 0 */
            }
        }
    }
    bool asph = has_asphere(s);
    for (int i = 0; i < nr; ++i) {
        double t = roots[i];
        V3 q = p + t * d;
        if (k1 * c * q.z > 1.0) continue; /* other branch of the quadric */
        if (asph) {
            /* Newton from this conic root: only the first on-branch root seeds it,
             * and only inside 1.1x the aperture's bounding radius (the polynomial
             * is meaningless far outside the mirror it describes). */
            if (t <= eps) continue;
            double rb = 1.1 * aperture_bound(s);
            if (q.x * q.x + q.y * q.y > rb * rb) return false;
            bool conv = false;
            for (int it = 0; it < 32; ++it) {
                V3 x = p + t * d;
                double rho = x.x * x.x + x.y * x.y;
                double z, slope;
                if (!sag_and_slope(s, rho, &z, &slope)) return false;
                double f = x.z - z;
                double fp = d.z - slope * 2.0 * (x.x * d.x + x.y * d.y);
                if (fp == 0.0) break;
                double dt = f / fp;
                t -= dt;
                if (std::fabs(dt) < newton_tol) {
                    conv = true;
                    break;
                }
            }
            if (!conv) {
                h->error = true;
                return false;
            }
            V3 x = p + t * d;
            double rho = x.x * x.x + x.y * x.y, z, slope;
            if (!sag_and_slope(s, rho, &z, &slope)) return false;
            if (t <= eps) return false;
            double m;
            bool in = aperture_inside(s, x.x, x.y, &m);
            cands->push_back(Cand{t, std::fabs(m)});
            if (!in) return false;
            h->t = t;
            h->pl = x;
            h->nl = normalize(v3(-2.0 * x.x * slope, -2.0 * x.y * slope, 1.0));
            return true;
        }
        if (t <= eps) continue;
        double m;
        bool in = aperture_inside(s, q.x, q.y, &m);
        cands->push_back(Cand{t, std::fabs(m)});
        if (!in) continue;
        h->t = t;
        h->pl = q;
        h->nl = normalize(v3(-c * q.x, -c * q.y, 1.0 - c * k1 * q.z));
        return true;
    }
    return false;
}

/* Finite open cylinder x^2 + y^2 = a^2, 0 <= z <= L (masts, Sec. 3). */
bool hit_cylinder(const o_surface& s, V3 p, V3 d, double eps, LocalHit* h, std::vector<Cand>* cands) {
    double rad = s.prm[0], len = s.prm[1];
    double a = d.x * d.x + d.y * d.y;
    if (a == 0.0) return false;
    double b = p.x * d.x + p.y * d.y;
    double g = p.x * p.x + p.y * p.y - rad * rad;
    double disc = b * b - a * g;
    if (disc < 0.0) return false;
    double sq = std::sqrt(disc);
    double q = -(b + (b >= 0.0 ? sq : -sq));
    double r[2];
    int nr = 0;
    if (q != 0.0) {
        r[0] = std::fmin(q / a, g / q);
        r[1] = std::fmax(q / a, g / q);
        nr = 2;
    } else {
        r[0] = 0.0;
        nr = 1;
    }
    for (int i = 0; i < nr; ++i) {
        double t = r[i];
        if (t <= eps) continue;
        V3 x = p + t * d;
        double m = std::fmin(x.z, len - x.z) / len;
        cands->push_back(Cand{t, std::fabs(m)});
        if (x.z < 0.0 || x.z > len) continue;
        h->t = t;
        h->pl = x;
        h->nl = normalize(v3(x.x, x.y, 0.0));
        return true;
    }
    return false;
}

/* Axis-aligned box |x| <= hx, |y| <= hy, |z| <= hz in the local frame. */
bool hit_box(const o_surface& s, V3 p, V3 d, double eps, LocalHit* h) {
    double pp[3] = {p.x, p.y, p.z}, dd[3] = {d.x, d.y, d.z};
    double tn = -INFINITY, tf = INFINITY;
    int axn = -1, axf = -1;
    for (int ax = 0; ax < 3; ++ax) {
        double hw = s.prm[ax];
        if (dd[ax] == 0.0) {
            if (std::fabs(pp[ax]) > hw) return false;
            continue;
        }
        double t1 = (-hw - pp[ax]) / dd[ax], t2 = (hw - pp[ax]) / dd[ax];
        double lo = std::fmin(t1, t2), hi = std::fmax(t1, t2);
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
    double t;
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
    h->t = t;
    h->pl = p + t * d;
    double nn[3] = {0, 0, 0};
    double comp = ax == 0 ? h->pl.x : (ax == 1 ? h->pl.y : h->pl.z);
    if (ax >= 0) nn[ax] = comp >= 0.0 ? 1.0 : -1.0;
    h->nl = v3(nn[0], nn[1], nn[2]);
    return true;
}

/* Hexagonal cone with a quadratic-Bezier wall profile (Sec. 2.2,
 * AGeoBezierPgon; the Winston cone AGeoWinstonConePoly is the special case
 * whose control points lie on a parabola).  Wall j (j = 0..5) is the set of
 * points whose coordinate along u_j = (cos j pi/3, sin j pi/3) equals the
 * profile radius r(u) at height z(u), with (r, z)(u) the Bezier curve
 * (1-u)^2 P0 + 2u(1-u) P1 + u^2 P2, u in [0, 1], and which lie in wall j's
 * 60-degree wedge (their u_j coordinate is the largest of the six).  In the
 * (q, z) half-plane of wall j, the ray is the line (q0 + t dq, z0 + t dz);
 * crossing the curve means dz (r(u) - q0) - dq (z(u) - z0) = 0, a quadratic in
 * u.  Front side = the side facing the cone axis. */
bool hit_hexcone(const o_surface& s, V3 p, V3 d, double eps, LocalHit* h, std::vector<Cand>* cands) {
    double r0 = s.prm[0], z0b = s.prm[1], r1 = s.prm[2], z1b = s.prm[3], r2 = s.prm[4], z2b = s.prm[5];
    double ra0 = r0, ra1 = 2.0 * (r1 - r0), ra2 = r0 - 2.0 * r1 + r2;
    double za0 = z0b, za1 = 2.0 * (z1b - z0b), za2 = z0b - 2.0 * z1b + z2b;
    bool found = false;
    for (int j = 0; j < 6; ++j) {
        double cj = std::cos(j * M_PI / 3.0), sj = std::sin(j * M_PI / 3.0);
        double q0 = p.x * cj + p.y * sj, dq = d.x * cj + d.y * sj;
        double den = dq * dq + d.z * d.z;
        if (den == 0.0) continue;
        double A = d.z * ra2 - dq * za2;
        double B = d.z * ra1 - dq * za1;
        double C = d.z * (ra0 - q0) - dq * (za0 - p.z);
        double us[2];
        int nu = 0;
        if (A == 0.0) {
            if (B != 0.0) us[nu++] = -C / B;
        } else {
            double disc = B * B - 4.0 * A * C;
            if (disc >= 0.0) {
                double sq = std::sqrt(disc);
                double q = -0.5 * (B + (B >= 0.0 ? sq : -sq));
                if (q != 0.0) {
                    us[nu++] = q / A;
                    us[nu++] = C / q;
                } else {
                    us[nu++] = -B / (2.0 * A);
                }
            }
        }
        for (int i = 0; i < nu; ++i) {
            double u = us[i];
            /* one Newton polish of the root */
            double gp = 2.0 * A * u + B;
            if (gp != 0.0) u -= ((A * u + B) * u + C) / gp;
            double R = ra0 + u * (ra1 + u * ra2);
            double Z = za0 + u * (za1 + u * za2);
            double t = ((R - q0) * dq + (Z - p.z) * d.z) / den;
            if (t <= eps) continue;
            V3 x = p + t * d;
            double qj = x.x * cj + x.y * sj;
            double qmax_other = -INFINITY;
            for (int m = 0; m < 6; ++m) {
                if (m == j) continue;
                double qm = x.x * std::cos(m * M_PI / 3.0) + x.y * std::sin(m * M_PI / 3.0);
                qmax_other = std::fmax(qmax_other, qm);
            }
            double rel = std::fmin((qj - qmax_other) / std::fmax(std::fabs(qj), 1e-300), std::fmin(u, 1.0 - u));
            if (u < 0.0 || u > 1.0) {
                cands->push_back(Cand{t, std::fabs(rel)});
                continue;
            }
            cands->push_back(Cand{t, std::fabs(rel)});
            if (qj < qmax_other) continue;
            if (found && !(t < h->t)) continue;
            double Rp = ra1 + 2.0 * ra2 * u, Zp = za1 + 2.0 * za2 * u;
            h->t = t;
            h->pl = x;
            h->nl = normalize(v3(-Zp * cj, -Zp * sj, Rp));
            found = true;
        }
    }
    return found;
}

struct Hit {
    bool any;
    bool error;
    double t;
    int sid;
    V3 pl;      /* local point */
    V3 nw;      /* world front normal */
    double margin;
};

bool intersect_surface(const o_surface& s, const Frame& f, V3 p, V3 d, double eps, double newton_tol,
                       LocalHit* lh, std::vector<Cand>* cands) {
    V3 pl = to_local_pt(f, p), dl = to_local_vec(f, d);
    lh->error = false;
    switch (s.shape) {
        case O_SHAPE_SAG: return hit_sag(s, pl, dl, eps, newton_tol, lh, cands);
        case O_SHAPE_CYLINDER: return hit_cylinder(s, pl, dl, eps, lh, cands);
        case O_SHAPE_BOX: return hit_box(s, pl, dl, eps, lh);
        case O_SHAPE_HEXCONE: return hit_hexcone(s, pl, dl, eps, lh, cands);
    }
    return false;
}

/* Reflectivity R(lambda): piecewise linear in the table, clamped at both ends. */
double reflectivity(const o_material& m, double lam) {
    if (m.n <= 1 || lam <= m.lam[0]) return m.refl[0];
    if (lam >= m.lam[m.n - 1]) return m.refl[m.n - 1];
    int i = 0;
    while (i + 1 < m.n - 1 && lam >= m.lam[i + 1]) ++i;
    double frac = (lam - m.lam[i]) / (m.lam[i + 1] - m.lam[i]);
    return m.refl[i] + (m.refl[i + 1] - m.refl[i]) * frac;
}

/* Sellmeier: n^2 = 1 + sum_i B_i l^2 / (l^2 - C_i), l in micrometres. */
double refr_index(const o_medium& m, double lam_nm) {
    if (m.n_const > 0.0) return m.n_const;
    double l2 = (lam_nm * 1e-3) * (lam_nm * 1e-3);
    double n2 = 1.0;
    for (int i = 0; i < 3; ++i) n2 += m.B[i] * l2 / (l2 - m.C[i]);
    return std::sqrt(n2);
}

/* Absorption length of a medium at lambda: piecewise linear in its table,
 * clamped; INFINITY without a table (no bulk absorption). */
double abs_length(const o_medium& m, double lam) {
    if (m.n_abs <= 0) return INFINITY;
    if (m.n_abs == 1 || lam <= m.abs_lam[0]) return m.abs_len[0];
    if (lam >= m.abs_lam[m.n_abs - 1]) return m.abs_len[m.n_abs - 1];
    int i = 0;
    while (i + 1 < m.n_abs - 1 && lam >= m.abs_lam[i + 1]) ++i;
    double frac = (lam - m.abs_lam[i]) / (m.abs_lam[i + 1] - m.abs_lam[i]);
    return m.abs_len[i] + (m.abs_len[i + 1] - m.abs_len[i]) * frac;
}

/* Unpolarised Fresnel reflectance: mean of |r_s|^2 and |r_p|^2; 1 under TIR. */
double fresnel(double n1, double n2, double cos_i) {
    double eta = n1 / n2;
    double sin2_t = eta * eta * (1.0 - cos_i * cos_i);
    if (sin2_t >= 1.0) return 1.0;
    double cos_t = std::sqrt(1.0 - sin2_t);
    double rs = (n1 * cos_i - n2 * cos_t) / (n1 * cos_i + n2 * cos_t);
    double rp = (n2 * cos_i - n1 * cos_t) / (n2 * cos_i + n1 * cos_t);
    return 0.5 * (rs * rs + rp * rp);
}

V3 reflect(V3 d, V3 n) { return d - (2.0 * dot(d, n)) * n; }

/* Orthonormal basis around a unit normal, Duff et al. 2017 (JCGT 6(1)). */
void onb(V3 n, V3* t, V3* b) {
    double sign = n.z >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (sign + n.z);
    double bb = n.x * n.y * a;
    *t = v3(1.0 + sign * n.x * n.x * a, sign * bb, -sign * n.x);
    *b = v3(bb, sign + n.y * n.y * a, -n.y);
}

struct Ctx {
    const o_scene* sc;
    std::vector<Frame> frames;
    double eps, newton_tol;
};

Hit nearest_hit(const Ctx& cx, int v, V3 p, V3 d) {
    const o_scene* sc = cx.sc;
    int s0 = 0, s1 = sc->n_surfaces;
    if (sc->variant_offsets) {
        s0 = sc->variant_offsets[v];
        s1 = sc->variant_offsets[v + 1];
    }
    Hit best;
    best.any = false;
    best.error = false;
    best.t = INFINITY;
    best.sid = -1;
    best.margin = INFINITY;
    std::vector<Cand> cands;
    for (int s = s0; s < s1; ++s) {
        LocalHit lh;
        bool ok = intersect_surface(sc->surfaces[s], cx.frames[s], p, d, cx.eps, cx.newton_tol, &lh, &cands);
        if (lh.error) best.error = true;
        if (!ok) continue;
        /* nearest t wins; equal t: the lower surface id (already in place) */
        if (lh.t < best.t) {
            best.any = true;
            best.t = lh.t;
            best.sid = s;
            best.pl = lh.pl;
            best.nw = to_world_vec(cx.frames[s], lh.nl);
        }
    }
    for (const Cand& c : cands)
        if (c.t <= best.t && c.margin < best.margin) best.margin = c.margin;
    return best;
}

/* One interaction of a recorded photon track (Fig. 2a shows such tracks). */
struct TrackRec {
    int64_t photon;
    int bounce, sid, status;
    V3 p;
};

void trace_range(const Ctx& cx, int64_t i0, int64_t i1, int64_t n, const double* O, const double* D,
                 const double* L, const int32_t* vop, uint64_t seed, int64_t first_id, int32_t max_bounces,
                 const o_outputs* out, std::vector<TrackRec>* track = nullptr) {
    const o_scene* sc = cx.sc;
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t i = i0; i < i1; ++i) {
        V3 p = v3(O[i], O[n + i], O[2 * n + i]);
        V3 d = v3(D[i], D[n + i], D[2 * n + i]);
        double lam = L[i];
        int v = vop ? vop[i] : 0;
        int64_t pid = first_id + i;
        int bounces = 0;
        int status = 0;
        int last = -1;
        double fx = 0.0, fy = 0.0;
        double margin = INFINITY;
        double cond = 0.0;  /* conditioning of the path: sum of 1 / |cos(incidence)| */
        while (status == 0) {
            Hit h = nearest_hit(cx, v, p, d);
            if (h.margin < margin) margin = h.margin;
            if (h.error) {
                status = O_ST_ERROR;
                break;
            }
            if (!h.any) {
                status = O_ST_ESCAPED;
                break;
            }
            p = p + h.t * d;
            last = h.sid;
            const o_surface& s = sc->surfaces[h.sid];
            uint32_t ctr[4] = {(uint32_t)pid, (uint32_t)((uint64_t)pid >> 32), (uint32_t)bounces, 0u};
            uint32_t w[4];
            philox(ctr, key, w);
            ++bounces;
            V3 n = h.nw;
            bool front = dot(d, n) < 0.0;
            cond += 1.0 / std::fmax(std::fabs(dot(d, n)), 1e-9);
            switch (s.role) {
                case O_ROLE_OBSCURATION: status = O_ST_OBSCURED; break;
                case O_ROLE_FOCAL:
                    if (front) {
                        status = O_ST_DETECTED;
                        fx = h.pl.x;
                        fy = h.pl.y;
                    } else {
                        status = O_ST_OBSCURED;
                    }
                    break;
                case O_ROLE_MIRROR: {
                    if (!front) {
                        status = O_ST_OBSCURED;
                        break;
                    }
                    const o_material& m = sc->materials[s.material];
                    double R = reflectivity(m, lam);
                    double thr = std::floor(R * 4294967296.0);
                    if (!((double)w[0] < thr)) {
                        status = O_ST_ABSORBED;
                        break;
                    }
                    V3 nn = n;
                    if (m.sigma > 0.0) {
                        double u1 = unit_open(w[1]), u2 = unit_open(w[2]);
                        double rad = std::sqrt(-2.0 * std::log(u1));
                        double g1 = rad * std::cos(2.0 * M_PI * u2);
                        double g2 = rad * std::sin(2.0 * M_PI * u2);
                        V3 t, b;
                        onb(n, &t, &b);
                        nn = normalize(n + (m.sigma * g1) * t + (m.sigma * g2) * b);
                    }
                    d = normalize(reflect(d, nn));
                    break;
                }
                case O_ROLE_REFRACT: {
                    /* bulk absorption over the segment just travelled, which lies in the
                     * medium on the photon's side of this face: survive with probability
                     * exp(-t / len(lambda)), draw u3 */
                    const o_medium& m_in = sc->media[front ? s.medium_front : s.medium_back];
                    const double len = abs_length(m_in, lam);
                    if (len < INFINITY) {
                        const double surv = std::exp(-h.t / len);
                        const double u3 = unit_open(w[3]);
                        const double am = std::fabs(u3 - surv);
                        if (am < margin) margin = am;
                        if (!(u3 < surv)) {
                            status = O_ST_ABSORBED;
                            break;
                        }
                    }
                    double na = refr_index(sc->media[s.medium_front], lam);
                    double nb = refr_index(sc->media[s.medium_back], lam);
                    double n1 = front ? na : nb, n2 = front ? nb : na;
                    V3 nf = front ? n : (-1.0) * n; /* normal facing the incoming photon */
                    double cos_i = -dot(d, nf);
                    double R = fresnel(n1, n2, cos_i);
                    double u0 = unit_open(w[0]);
                    if (std::fabs(u0 - R) < margin) margin = std::fabs(u0 - R);
                    if (u0 < R) {
                        d = normalize(reflect(d, nf));
                    } else {
                        double eta = n1 / n2;
                        double sin2_t = eta * eta * (1.0 - cos_i * cos_i);
                        double cos_t = std::sqrt(1.0 - sin2_t);
                        d = normalize(eta * d + (eta * cos_i - cos_t) * nf);
                    }
                    break;
                }
                default: status = O_ST_ERROR; break;
            }
            if (status == 0 && !(std::isfinite(d.x) && std::isfinite(d.y) && std::isfinite(d.z)))
                status = O_ST_ERROR;
            if (status == 0 && bounces >= max_bounces) status = O_ST_MAX_BOUNCES;
            if (track) track->push_back(TrackRec{i, bounces - 1, last, status, p});
        }
        out->status[i] = (uint8_t)status;
        out->bounces[i] = (uint8_t)bounces;
        if (out->hit) {
            out->hit[i] = p.x;
            out->hit[n + i] = p.y;
            out->hit[2 * n + i] = p.z;
        }
        if (out->dir) {
            out->dir[i] = d.x;
            out->dir[n + i] = d.y;
            out->dir[2 * n + i] = d.z;
        }
        if (out->last_surface) out->last_surface[i] = last;
        if (out->focal_xy) {
            out->focal_xy[i] = fx;
            out->focal_xy[n + i] = fy;
        }
        if (out->edge_margin) out->edge_margin[i] = margin;
        if (out->cond) out->cond[i] = cond;
    }
}

int check_scene(const o_scene* sc) {
    if (!sc || sc->n_surfaces <= 0 || !sc->surfaces) return -1;
    for (int s = 0; s < sc->n_surfaces; ++s) {
        const o_surface& su = sc->surfaces[s];
        if (su.shape < 0 || su.shape > 3 || su.role < 0 || su.role > 3) return -2;
        if (su.role == O_ROLE_MIRROR && (su.material < 0 || su.material >= sc->n_materials)) return -3;
        if (su.role == O_ROLE_REFRACT &&
            (su.medium_front < 0 || su.medium_front >= sc->n_media || su.medium_back < 0 ||
             su.medium_back >= sc->n_media))
            return -4;
    }
    return 0;
}


/* ==================================================== frozen-path gradients
 * Forward-mode dual numbers: every quantity carries its value and its
 * derivatives with respect to up to NT parameters: the parameters of up to
 * NSURF differentiable surfaces of a photon's path (10 slots each, see
 * oracle.h).  A path that meets more of them is replayed once per group of
 * NSURF surfaces. */
constexpr int NSURF = 4;
constexpr int NT = 10 * NSURF;

struct Dual {
    double v;
    double d[NT];
};
Dual dconst(double v) {
    Dual r;
    r.v = v;
    for (int k = 0; k < NT; ++k) r.d[k] = 0.0;
    return r;
}
Dual operator+(const Dual& a, const Dual& b) {
    Dual r;
    r.v = a.v + b.v;
    for (int k = 0; k < NT; ++k) r.d[k] = a.d[k] + b.d[k];
    return r;
}
Dual operator-(const Dual& a, const Dual& b) {
    Dual r;
    r.v = a.v - b.v;
    for (int k = 0; k < NT; ++k) r.d[k] = a.d[k] - b.d[k];
    return r;
}
Dual operator-(const Dual& a) {
    Dual r;
    r.v = -a.v;
    for (int k = 0; k < NT; ++k) r.d[k] = -a.d[k];
    return r;
}
Dual operator*(const Dual& a, const Dual& b) {
    Dual r;
    r.v = a.v * b.v;
    for (int k = 0; k < NT; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
Dual operator/(const Dual& a, const Dual& b) {
    Dual r;
    r.v = a.v / b.v;
    for (int k = 0; k < NT; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) / b.v;
    return r;
}
Dual operator+(const Dual& a, double b) { return a + dconst(b); }
Dual operator+(double a, const Dual& b) { return dconst(a) + b; }
Dual operator-(const Dual& a, double b) { return a - dconst(b); }
Dual operator-(double a, const Dual& b) { return dconst(a) - b; }
Dual operator*(const Dual& a, double b) { return a * dconst(b); }
Dual operator*(double a, const Dual& b) { return dconst(a) * b; }
Dual operator/(const Dual& a, double b) { return a / dconst(b); }
Dual operator/(double a, const Dual& b) { return dconst(a) / b; }

double val(double x) { return x; }
double val(const Dual& x) { return x.v; }
double nsqrt(double x) { return std::sqrt(x); }
Dual nsqrt(const Dual& x) {
    Dual r;
    r.v = std::sqrt(x.v);
    for (int k = 0; k < NT; ++k) r.d[k] = x.d[k] / (2.0 * r.v);
    return r;
}
double ncos(double x) { return std::cos(x); }
double nsin(double x) { return std::sin(x); }
Dual ncos(const Dual& x) {
    Dual r;
    r.v = std::cos(x.v);
    const double s = -std::sin(x.v);
    for (int k = 0; k < NT; ++k) r.d[k] = s * x.d[k];
    return r;
}
Dual nsin(const Dual& x) {
    Dual r;
    r.v = std::sin(x.v);
    const double c = std::cos(x.v);
    for (int k = 0; k < NT; ++k) r.d[k] = c * x.d[k];
    return r;
}
template <class N>
N nlit(double v);
template <>
double nlit<double>(double v) { return v; }
template <>
Dual nlit<Dual>(double v) { return dconst(v); }

template <class N>
struct NV3 {
    N x, y, z;
};
template <class N>
NV3<N> nv3(N x, N y, N z) { return NV3<N>{x, y, z}; }
template <class N>
NV3<N> operator+(const NV3<N>& a, const NV3<N>& b) { return nv3<N>(a.x + b.x, a.y + b.y, a.z + b.z); }
template <class N>
NV3<N> operator-(const NV3<N>& a, const NV3<N>& b) { return nv3<N>(a.x - b.x, a.y - b.y, a.z - b.z); }
template <class N>
NV3<N> scale(const N& s, const NV3<N>& a) { return nv3<N>(s * a.x, s * a.y, s * a.z); }
template <class N>
N ndot(const NV3<N>& a, const NV3<N>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class N>
NV3<N> nunit(const NV3<N>& a) { return scale<N>(1.0 / nsqrt(ndot(a, a)), a); }

/* The surface with its parameters as numbers of type N. */
template <class N>
struct PSurf {
    const o_surface* s;
    N rows[9];  /* tilted frame */
    N asph[8];
    N bz[6];    /* Bezier control points (r, z) x 3 */
};

/* params: 16 numbers in the layout of oracle.h */
template <class N>
PSurf<N> make_psurf(const o_surface& s, const N* prm) {
    PSurf<N> P;
    P.s = &s;
    const N ca = ncos(prm[0]), sa = nsin(prm[0]);
    const N cb = ncos(prm[1]), sb = nsin(prm[1]);
    const N z0 = nlit<N>(0.0), one = nlit<N>(1.0);
    const N rxT[9] = {one, z0, z0, z0, ca, sa, z0, -sa, ca};
    const N ryT[9] = {cb, z0, -sb, z0, one, z0, sb, z0, cb};
    N tmp[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            N acc = nlit<N>(0.0);
            for (int k = 0; k < 3; ++k) acc = acc + rxT[3 * i + k] * s.rot[3 * k + j];
            tmp[3 * i + j] = acc;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            N acc = nlit<N>(0.0);
            for (int k = 0; k < 3; ++k) acc = acc + ryT[3 * i + k] * tmp[3 * k + j];
            P.rows[3 * i + j] = acc;
        }
    for (int k = 0; k < 8; ++k) P.asph[k] = prm[2 + k];
    for (int k = 0; k < 6; ++k) P.bz[k] = prm[10 + k];
    return P;
}

template <class N>
NV3<N> p_local_pt(const PSurf<N>& P, const NV3<N>& p) {
    const NV3<N> q = nv3<N>(p.x - P.s->origin[0], p.y - P.s->origin[1], p.z - P.s->origin[2]);
    return nv3<N>(P.rows[0] * q.x + P.rows[1] * q.y + P.rows[2] * q.z, P.rows[3] * q.x + P.rows[4] * q.y + P.rows[5] * q.z,
                  P.rows[6] * q.x + P.rows[7] * q.y + P.rows[8] * q.z);
}
template <class N>
NV3<N> p_local_vec(const PSurf<N>& P, const NV3<N>& q) {
    return nv3<N>(P.rows[0] * q.x + P.rows[1] * q.y + P.rows[2] * q.z, P.rows[3] * q.x + P.rows[4] * q.y + P.rows[5] * q.z,
                  P.rows[6] * q.x + P.rows[7] * q.y + P.rows[8] * q.z);
}
template <class N>
NV3<N> p_world_vec(const PSurf<N>& P, const NV3<N>& q) {
    return nv3<N>(P.rows[0] * q.x + P.rows[3] * q.y + P.rows[6] * q.z, P.rows[1] * q.x + P.rows[4] * q.y + P.rows[7] * q.z,
                  P.rows[2] * q.x + P.rows[5] * q.y + P.rows[8] * q.z);
}

/* sag and dsag/drho with the surface's conic and the parameter asphere */
template <class N>
bool p_sag(const PSurf<N>& P, const N& rho, N* z, N* slope) {
    const double c = P.s->curv, k1 = 1.0 + P.s->conic;
    const N arg = 1.0 - k1 * c * c * rho;
    if (val(arg) < 0.0) return false;
    const N sq = nsqrt(arg);
    N zz = c * rho / (1.0 + sq), sl = c / (2.0 * sq);
    N rp = rho, rpm = nlit<N>(1.0);
    for (int i = 1; i <= 8; ++i) {
        zz = zz + P.asph[i - 1] * rp;
        sl = sl + (double)i * P.asph[i - 1] * rpm;
        rpm = rp;
        rp = rp * rho;
    }
    *z = zz;
    *slope = sl;
    return true;
}

/* Re-intersect a recorded SAG surface: conic roots, the on-branch root
 * nearest the recorded distance t0, then Newton on the full sag (value
 * converged, plus one step so the derivatives are those of the exact root). */
template <class N>
bool p_hit_sag(const PSurf<N>& P, const NV3<N>& p, const NV3<N>& d, double t0, N* t, NV3<N>* pl, NV3<N>* nl) {
    const double c = P.s->curv, k1 = 1.0 + P.s->conic;
    const N a = c * (d.x * d.x + d.y * d.y + k1 * d.z * d.z);
    const N b = c * (p.x * d.x + p.y * d.y + k1 * p.z * d.z) - d.z;
    const N g = c * (p.x * p.x + p.y * p.y + k1 * p.z * p.z) - 2.0 * p.z;
    N roots[2];
    int nr = 0;
    if (val(a) == 0.0) {
        if (val(b) != 0.0) roots[nr++] = -g / (2.0 * b);
    } else {
        const N disc = b * b - a * g;
        if (val(disc) >= 0.0) {
            const N sq = nsqrt(disc);
            const N q = -(b + (val(b) >= 0.0 ? sq : -sq));
            if (val(q) != 0.0) {
                roots[nr++] = q / a;
                roots[nr++] = g / q;
            } else {
                roots[nr++] = nlit<N>(0.0) * b;
            }
        }
    }
    int best = -1;
    for (int i = 0; i < nr; ++i) {
        const NV3<N> x = p + scale<N>(roots[i], d);
        if (k1 * c * val(x.z) > 1.0) continue;
        if (best < 0 || std::fabs(val(roots[i]) - t0) < std::fabs(val(roots[best]) - t0)) best = i;
    }
    N tt = best >= 0 ? roots[best] : nlit<N>(t0) + nlit<N>(0.0) * a;
    for (int it = 0; it < 40; ++it) {
        const NV3<N> x = p + scale<N>(tt, d);
        N z, sl;
        if (!p_sag(P, x.x * x.x + x.y * x.y, &z, &sl)) return false;
        const N f = x.z - z;
        const N fp = d.z - sl * 2.0 * (x.x * d.x + x.y * d.y);
        const N dt = f / fp;
        tt = tt - dt;
        if (std::fabs(val(dt)) < 1e-15 * (1.0 + std::fabs(val(tt))) && it > 0) break;
    }
    const NV3<N> x = p + scale<N>(tt, d);
    N z, sl;
    if (!p_sag(P, x.x * x.x + x.y * x.y, &z, &sl)) return false;
    *t = tt;
    *pl = x;
    *nl = nunit(nv3<N>(-2.0 * x.x * sl, -2.0 * x.y * sl, nlit<N>(1.0)));
    return true;
}

/* Re-intersect a recorded Bezier hex cone: the wall/root whose distance is
 * nearest the recorded one. */
template <class N>
bool p_hit_hexcone(const PSurf<N>& P, const NV3<N>& p, const NV3<N>& d, double t0, N* t, NV3<N>* pl, NV3<N>* nl) {
    const N ra0 = P.bz[0], ra1 = 2.0 * (P.bz[2] - P.bz[0]), ra2 = P.bz[0] - 2.0 * P.bz[2] + P.bz[4];
    const N za0 = P.bz[1], za1 = 2.0 * (P.bz[3] - P.bz[1]), za2 = P.bz[1] - 2.0 * P.bz[3] + P.bz[5];
    bool found = false;
    double bestd = INFINITY;
    for (int j = 0; j < 6; ++j) {
        const double cj = std::cos(j * M_PI / 3.0), sj = std::sin(j * M_PI / 3.0);
        const N q0 = p.x * cj + p.y * sj, dq = d.x * cj + d.y * sj;
        const N den = dq * dq + d.z * d.z;
        if (val(den) == 0.0) continue;
        const N A = d.z * ra2 - dq * za2, B = d.z * ra1 - dq * za1, C = d.z * (ra0 - q0) - dq * (za0 - p.z);
        N us[2];
        int nu = 0;
        if (val(A) == 0.0) {
            if (val(B) != 0.0) us[nu++] = -C / B;
        } else {
            const N disc = B * B - 4.0 * A * C;
            if (val(disc) >= 0.0) {
                const N sq = nsqrt(disc);
                const N q = -0.5 * (B + (val(B) >= 0.0 ? sq : -sq));
                if (val(q) != 0.0) {
                    us[nu++] = q / A;
                    us[nu++] = C / q;
                } else {
                    us[nu++] = -B / (2.0 * A);
                }
            }
        }
        for (int i = 0; i < nu; ++i) {
            N u = us[i];
            const N gp = 2.0 * A * u + B;
            if (val(gp) != 0.0) u = u - ((A * u + B) * u + C) / gp;
            const N R = ra0 + u * (ra1 + u * ra2), Z = za0 + u * (za1 + u * za2);
            const N tt = ((R - q0) * dq + (Z - p.z) * d.z) / den;
            const double dist = std::fabs(val(tt) - t0);
            if (dist < bestd) {
                bestd = dist;
                found = true;
                *t = tt;
                *pl = p + scale<N>(tt, d);
                const N Rp = ra1 + 2.0 * ra2 * u, Zp = za1 + 2.0 * za2 * u;
                *nl = nunit(nv3<N>(-Zp * cj, -Zp * sj, Rp));
            }
        }
    }
    return found;
}

enum { ACT_REFLECT = 0, ACT_REFRACT = 1, ACT_DETECT = 2, ACT_STOP = 3 };
struct Step {
    int sid, act;
    double t;
};

/* Nominal trace in expected-weight mode, recording the path. */
int record_path(const Ctx& cx, int v, V3 p, V3 d, double lam, int64_t pid, const uint32_t key[2], int max_bounces,
                std::vector<Step>* path, double* w) {
    const o_scene* sc = cx.sc;
    *w = 1.0;
    path->clear();
    int bounces = 0;
    while (true) {
        Hit h = nearest_hit(cx, v, p, d);
        if (h.error) return O_ST_ERROR;
        if (!h.any) return O_ST_ESCAPED;
        p = p + h.t * d;
        const o_surface& s = sc->surfaces[h.sid];
        uint32_t ctr[4] = {(uint32_t)pid, (uint32_t)((uint64_t)pid >> 32), (uint32_t)bounces, 0u};
        uint32_t wd[4];
        philox(ctr, key, wd);
        ++bounces;
        V3 n = h.nw;
        bool front = dot(d, n) < 0.0;
        Step st{h.sid, ACT_STOP, h.t};
        if (s.role == O_ROLE_OBSCURATION) {
            path->push_back(st);
            return O_ST_OBSCURED;
        }
        if (s.role == O_ROLE_FOCAL) {
            st.act = front ? ACT_DETECT : ACT_STOP;
            path->push_back(st);
            return front ? O_ST_DETECTED : O_ST_OBSCURED;
        }
        if (s.role == O_ROLE_MIRROR) {
            if (!front) {
                path->push_back(st);
                return O_ST_OBSCURED;
            }
            const o_material& m = sc->materials[s.material];
            *w *= reflectivity(m, lam);
            V3 nn = n;
            if (m.sigma > 0.0) {
                double u1 = unit_open(wd[1]), u2 = unit_open(wd[2]);
                double rad = std::sqrt(-2.0 * std::log(u1));
                V3 t, b;
                onb(n, &t, &b);
                nn = normalize(n + (m.sigma * rad * std::cos(2.0 * M_PI * u2)) * t +
                               (m.sigma * rad * std::sin(2.0 * M_PI * u2)) * b);
            }
            d = normalize(reflect(d, nn));
            st.act = ACT_REFLECT;
        } else {
            /* expected-weight mode: bulk absorption multiplies the weight */
            const double len = abs_length(sc->media[front ? s.medium_front : s.medium_back], lam);
            if (len < INFINITY) *w *= std::exp(-h.t / len);
            double na = refr_index(sc->media[s.medium_front], lam), nb = refr_index(sc->media[s.medium_back], lam);
            double n1 = front ? na : nb, n2 = front ? nb : na;
            V3 nf = front ? n : (-1.0) * n;
            double ci = -dot(d, nf);
            if (unit_open(wd[0]) < fresnel(n1, n2, ci)) {
                d = normalize(reflect(d, nf));
                st.act = ACT_REFLECT;
            } else {
                double eta = n1 / n2, s2 = eta * eta * (1.0 - ci * ci);
                d = normalize(eta * d + (eta * ci - std::sqrt(1.0 - s2)) * nf);
                st.act = ACT_REFRACT;
            }
        }
        path->push_back(st);
        if (bounces >= max_bounces) return O_ST_MAX_BOUNCES;
    }
}

bool differentiable(const o_surface& s) {
    return s.role == O_ROLE_MIRROR && (s.shape == O_SHAPE_SAG || s.shape == O_SHAPE_HEXCONE);
}

/* The differentiable surfaces whose parameters carry derivative slots in one
 * replay: surface sid[j] owns slots 10 j .. 10 j + 9. */
struct Tracked {
    int sid[NSURF];
    int n = 0;
    int index(int s) const {
        for (int j = 0; j < n; ++j)
            if (sid[j] == s) return j;
        return -1;
    }
};

/* Replay one recorded path with parameters as numbers of type N; the
 * parameters of the `tracked` surfaces carry derivative slots (Dual only). */
template <class N>
struct Replay {
    bool ok;
    NV3<N> p, d;  /* final point and direction */
    N qx, qy;     /* focal-surface local point (DETECTED) */
};

template <class N>
N param_number(double v, int slot);
template <>
double param_number<double>(double v, int) { return v; }
template <>
Dual param_number<Dual>(double v, int slot) {
    Dual r = dconst(v);
    if (slot >= 0 && slot < NT) r.d[slot] = 1.0;
    return r;
}

template <class N>
PSurf<N> psurf_for(const o_surface& s, int sid, const Tracked& tracked, const double* delta) {
    N prm[O_N_PARAM];
    double nom[O_N_PARAM];
    nom[0] = s.tilt[0];
    nom[1] = s.tilt[1];
    for (int k = 0; k < 8; ++k) nom[2 + k] = s.asph[k];
    for (int k = 0; k < 6; ++k) nom[10 + k] = s.prm[k];
    for (int k = 0; k < O_N_PARAM; ++k) {
        const double v = nom[k] + (delta ? delta[(size_t)sid * O_N_PARAM + k] : 0.0);
        int slot = -1;
        const int j = tracked.index(sid);
        if (j >= 0) {
            const int local = s.shape == O_SHAPE_SAG ? (k < 10 ? k : -1) : (k >= 10 ? k - 10 : -1);
            if (local >= 0) slot = 10 * j + local;
        }
        prm[k] = param_number<N>(v, slot);
    }
    return make_psurf<N>(s, prm);
}

template <class N>
Replay<N> replay(const Ctx& cx, const std::vector<Step>& path, V3 p0, V3 d0, double lam, int64_t pid,
                 const uint32_t key[2], const Tracked& tracked, const double* delta) {
    const o_scene* sc = cx.sc;
    Replay<N> R;
    R.ok = true;
    NV3<N> p = nv3<N>(nlit<N>(p0.x), nlit<N>(p0.y), nlit<N>(p0.z));
    NV3<N> d = nv3<N>(nlit<N>(d0.x), nlit<N>(d0.y), nlit<N>(d0.z));
    R.qx = nlit<N>(0.0);
    R.qy = nlit<N>(0.0);
    for (size_t b = 0; b < path.size(); ++b) {
        const Step& st = path[b];
        const o_surface& s = sc->surfaces[st.sid];
        const PSurf<N> P = psurf_for<N>(s, st.sid, tracked, delta);
        const NV3<N> pl = p_local_pt(P, p), dl = p_local_vec(P, d);
        N t;
        NV3<N> xl, nl;
        bool ok = false;
        if (s.shape == O_SHAPE_SAG) ok = p_hit_sag(P, pl, dl, st.t, &t, &xl, &nl);
        else if (s.shape == O_SHAPE_HEXCONE) ok = p_hit_hexcone(P, pl, dl, st.t, &t, &xl, &nl);
        else ok = false;
        if (!ok) {
            R.ok = false;
            return R;
        }
        p = p + scale<N>(t, d);
        if (st.act == ACT_DETECT) {
            R.qx = xl.x;
            R.qy = xl.y;
            break;
        }
        if (st.act == ACT_STOP) break;
        const NV3<N> n = p_world_vec(P, nl);
        const bool front = val(ndot(d, n)) < 0.0;
        uint32_t ctr[4] = {(uint32_t)pid, (uint32_t)((uint64_t)pid >> 32), (uint32_t)b, 0u};
        uint32_t wd[4];
        philox(ctr, key, wd);
        if (s.role == O_ROLE_MIRROR) {
            const o_material& m = sc->materials[s.material];
            NV3<N> nn = n;
            if (m.sigma > 0.0) {
                const double u1 = unit_open(wd[1]), u2 = unit_open(wd[2]);
                const double rad = std::sqrt(-2.0 * std::log(u1));
                const double g1 = rad * std::cos(2.0 * M_PI * u2), g2 = rad * std::sin(2.0 * M_PI * u2);
                const double sign = val(n.z) >= 0.0 ? 1.0 : -1.0;
                const N a = -1.0 / (sign + n.z);
                const N bb = n.x * n.y * a;
                const NV3<N> tt = nv3<N>(1.0 + sign * n.x * n.x * a, sign * bb, -sign * n.x);
                const NV3<N> bv = nv3<N>(bb, sign + n.y * n.y * a, -n.y);
                nn = nunit(n + scale<N>(nlit<N>(m.sigma * g1), tt) + scale<N>(nlit<N>(m.sigma * g2), bv));
            }
            d = nunit(d - scale<N>(2.0 * ndot(d, nn), nn));
        } else {
            const double na = refr_index(sc->media[s.medium_front], lam);
            const double nb = refr_index(sc->media[s.medium_back], lam);
            const double n1 = front ? na : nb, n2 = front ? nb : na;
            const NV3<N> nf = front ? n : scale<N>(nlit<N>(-1.0), n);
            if (st.act == ACT_REFLECT) {
                d = nunit(d - scale<N>(2.0 * ndot(d, nf), nf));
            } else {
                const double eta = n1 / n2;
                const N ci = -ndot(d, nf);
                const N s2 = eta * eta * (1.0 - ci * ci);
                d = nunit(scale<N>(nlit<N>(eta), d) + scale<N>(eta * ci - nsqrt(1.0 - s2), nf));
            }
        }
    }
    R.p = p;
    R.d = d;
    return R;
}

/* signed hexagon margin of the last segment's crossing of the variant's focal plane */
template <class N>
bool exit_margin(const o_scene* sc, int v, const NV3<N>& p, const NV3<N>& d, N* m) {
    int s0 = 0, s1 = sc->n_surfaces;
    if (sc->variant_offsets) {
        s0 = sc->variant_offsets[v];
        s1 = sc->variant_offsets[v + 1];
    }
    for (int s = s0; s < s1; ++s) {
        const o_surface& f = sc->surfaces[s];
        if (f.role != O_ROLE_FOCAL || f.shape != O_SHAPE_SAG || f.aperture != O_AP_HEXAGON) continue;
        const N zero[O_N_PARAM] = {};
        N prm[O_N_PARAM];
        for (int k = 0; k < O_N_PARAM; ++k) prm[k] = nlit<N>(0.0);
        prm[0] = nlit<N>(f.tilt[0]);
        prm[1] = nlit<N>(f.tilt[1]);
        (void)zero;
        const PSurf<N> P = make_psurf<N>(f, prm);
        const NV3<N> pl = p_local_pt(P, p), dl = p_local_vec(P, d);
        if (!(val(dl.z) < 0.0)) return false;
        const N t = -pl.z / dl.z;
        const NV3<N> x = pl + scale<N>(t, dl);
        const double s60 = std::sqrt(3.0) / 2.0;
        const N c0 = x.x, c1 = 0.5 * x.x + s60 * x.y, c2 = -0.5 * x.x + s60 * x.y;
        const N cand[3] = {c0, c1, c2};
        int km = 0;
        for (int k = 1; k < 3; ++k)
            if (std::fabs(val(cand[k])) > std::fabs(val(cand[km]))) km = k;
        const N mk = val(cand[km]) >= 0.0 ? cand[km] : -cand[km];
        *m = f.ap[0] - mk;
        return true;
    }
    return false;
}

double sigmoid(double x) { return 1.0 / (1.0 + std::exp(-x)); }
}  // namespace

extern "C" {

/* Source bundles of the batched concentrator study (uniform over the entrance
 * hexagon, Sec. 3 / Fig. 2b): rejection sampling in the bounding rectangle
 * [-a, a] x [-R, R], R = 2a / sqrt(3); candidate k of photon id uses Philox
 * counter (id_lo, id_hi, k, 1): x = (2 u0 - 1) a, y = (2 u1 - 1) R, accepted
 * iff max(|x|, |x/2 + s y|, |-x/2 + s y|) <= a with s = sqrt(3)/2; the
 * wavelength is lam_min + (lam_max - lam_min) u2 of the accepted draw. */
int64_t oracle_generate_sources(const o_source_group* groups, int32_t n_groups, uint64_t seed,
                                int64_t first_photon_id, double* O, double* D, double* L, int32_t* V) {
    int64_t n = 0;
    for (int g = 0; g < n_groups; ++g) n = std::max<int64_t>(n, groups[g].first + groups[g].n);
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    const double s60 = std::sqrt(3.0) / 2.0;
    int64_t failed = 0;
    for (int g = 0; g < n_groups; ++g) {
        const o_source_group& G = groups[g];
        const double a = G.apothem, R = G.apothem * 2.0 / std::sqrt(3.0);
        for (int64_t j = 0; j < G.n; ++j) {
            const int64_t i = G.first + j;
            const int64_t pid = first_photon_id + i;
            bool ok = false;
            double x = NAN, y = NAN, lam = NAN;
            for (uint32_t k = 0; k < 64 && !ok; ++k) {
                const uint32_t ctr[4] = {(uint32_t)pid, (uint32_t)((uint64_t)pid >> 32), k, 1u};
                uint32_t w[4];
                philox(ctr, key, w);
                const double cx = (2.0 * unit_open(w[0]) - 1.0) * a;
                const double cy = (2.0 * unit_open(w[1]) - 1.0) * R;
                const double m = std::fmax(std::fabs(cx), std::fmax(std::fabs(0.5 * cx + s60 * cy),
                                                                    std::fabs(-0.5 * cx + s60 * cy)));
                if (m <= a) {
                    ok = true;
                    x = cx;
                    y = cy;
                    lam = G.lam_min + (G.lam_max - G.lam_min) * unit_open(w[2]);
                }
            }
            if (!ok) ++failed;
            O[i] = G.c[0] + x;
            O[n + i] = G.c[1] + y;
            O[2 * n + i] = G.c[2];
            for (int c = 0; c < 3; ++c) D[c * n + i] = G.dir[c];
            L[i] = lam;
            V[i] = G.variant;
        }
    }
    return failed;
}


int oracle_objective(const o_scene* scene, int64_t n, const double* O, const double* D, const double* L,
                     const int32_t* vop, uint64_t seed, int64_t first_photon_id, int32_t max_bounces, double eps,
                     int32_t n_threads, int32_t objective, double tau, const double* delta, double* value,
                     double* grad) {
    int rc = check_scene(scene);
    if (rc) return rc;
    if (n <= 0 || max_bounces <= 0 || max_bounces > 255 || !value || objective < 0 || objective > 3) return -10;
    /* objectives 2 and 3 (pins only): w-weighted centroid x, y of the DETECTED photons */
    const bool centroid = objective >= 2;
    const int cax = objective - 2;
    Ctx cx;
    cx.sc = scene;
    cx.frames.resize(scene->n_surfaces);
    for (int s = 0; s < scene->n_surfaces; ++s) cx.frames[s] = make_frame(scene->surfaces[s]);
    cx.eps = eps;
    cx.newton_tol = eps * 1e-4;
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    if (n_threads <= 0) n_threads = 1;
    if ((int64_t)n_threads > n) n_threads = (int32_t)n;
    const size_t NP = (size_t)scene->n_surfaces * O_N_PARAM;
    // per photon: value-pass results; has_diff: the path meets a differentiable surface
    std::vector<int> status(n);
    std::vector<char> has_diff(n, 0);
    std::vector<double> w(n, 0.0), qx(n, 0.0), qy(n, 0.0), mval(n, 0.0);
    std::vector<char> valid(n, 0);
    auto photon = [&](int64_t i, std::vector<Step>& path) {
        V3 p = v3(O[i], O[n + i], O[2 * n + i]), d = v3(D[i], D[n + i], D[2 * n + i]);
        const int v = vop ? vop[i] : 0;
        const int64_t pid = first_photon_id + i;
        status[i] = record_path(cx, v, p, d, L[i], pid, key, max_bounces, &path, &w[i]);
        for (const Step& st : path)
            if (differentiable(scene->surfaces[st.sid])) has_diff[i] = 1;
    };
    // pass 1: values with the perturbed parameters
    {
        std::vector<std::thread> th;
        for (int k = 0; k < n_threads; ++k)
            th.emplace_back([&, k]() {
                std::vector<Step> path;
                for (int64_t i = n * k / n_threads; i < n * (k + 1) / n_threads; ++i) {
                    photon(i, path);
                    V3 p = v3(O[i], O[n + i], O[2 * n + i]), d = v3(D[i], D[n + i], D[2 * n + i]);
                    Replay<double> R = replay<double>(cx, path, p, d, L[i], first_photon_id + i, key, Tracked(), delta);
                    if (!R.ok) continue;
                    valid[i] = 1;
                    qx[i] = R.qx;
                    qy[i] = R.qy;
                    if (objective == 1 && status[i] != O_ST_OBSCURED && status[i] != O_ST_ERROR &&
                        status[i] != O_ST_MAX_BOUNCES) {
                        double m;
                        if (exit_margin<double>(scene, vop ? vop[i] : 0, R.p, R.d, &m)) mval[i] = m;
                        else valid[i] = 2;  // heading away: contributes 0
                    } else if (objective == 1) {
                        valid[i] = 2;
                    }
                }
            });
        for (auto& t : th) t.join();
    }
    /* per-variant sums; with several variants the objective is the sum of the
     * variants' objectives, each over its own photons */
    const int nvar = scene->variant_offsets ? scene->n_variants : 1;
    std::vector<double> Wv(nvar, 0.0), cxv(nvar, 0.0), cyv(nvar, 0.0), nv(nvar, 0.0);
    for (int64_t i = 0; i < n; ++i) {
        const int v = vop ? vop[i] : 0;
        nv[v] += 1.0;
        if (valid[i] == 1 && status[i] == O_ST_DETECTED) {
            Wv[v] += w[i];
            cxv[v] += w[i] * qx[i];
            cyv[v] += w[i] * qy[i];
        }
    }
    for (int v = 0; v < nvar; ++v)
        if (Wv[v] > 0.0) {
            cxv[v] /= Wv[v];
            cyv[v] /= Wv[v];
        }
    std::vector<double> part_v(nvar, 0.0);
    for (int64_t i = 0; i < n; ++i) {
        const int v = vop ? vop[i] : 0;
        if (valid[i] != 1) continue;
        if (objective == 1) {
            part_v[v] += w[i] * sigmoid(mval[i] / tau);
        } else if (status[i] == O_ST_DETECTED) {
            if (centroid) part_v[v] += w[i] * (cax == 0 ? qx[i] : qy[i]);
            else part_v[v] += w[i] * ((qx[i] - cxv[v]) * (qx[i] - cxv[v]) + (qy[i] - cyv[v]) * (qy[i] - cyv[v]));
        }
    }
    double total = 0.0;
    for (int v = 0; v < nvar; ++v) {
        if (objective == 1) {
            if (nv[v] > 0.0) total += part_v[v] / nv[v];
        } else if (Wv[v] > 0.0) {
            total += part_v[v] / Wv[v];
        }
    }
    *value = total;
    if (!grad) return 0;
    // pass 2: dual numbers along the same frozen paths, one thread-partial vector each
    std::vector<std::vector<double>> part(n_threads, std::vector<double>(NP, 0.0));
    {
        std::vector<std::thread> th;
        for (int k = 0; k < n_threads; ++k)
            th.emplace_back([&, k]() {
                std::vector<Step> path;
                std::vector<double>& g = part[k];
                double dummy_w;
                for (int64_t i = n * k / n_threads; i < n * (k + 1) / n_threads; ++i) {
                    if (valid[i] != 1 || !has_diff[i]) continue;
                    if (objective != 1 && status[i] != O_ST_DETECTED) continue;
                    V3 p = v3(O[i], O[n + i], O[2 * n + i]), d = v3(D[i], D[n + i], D[2 * n + i]);
                    const int v = vop ? vop[i] : 0;
                    record_path(cx, v, p, d, L[i], first_photon_id + i, key, max_bounces, &path, &dummy_w);
                    // every differentiable surface of the path, in order of first meeting
                    std::vector<int> sids;
                    for (const Step& st : path)
                        if (differentiable(scene->surfaces[st.sid]) &&
                            std::find(sids.begin(), sids.end(), st.sid) == sids.end())
                            sids.push_back(st.sid);
                    for (size_t g0 = 0; g0 < sids.size(); g0 += NSURF) {
                        Tracked tr;
                        for (size_t j = g0; j < sids.size() && tr.n < NSURF; ++j) tr.sid[tr.n++] = sids[j];
                        Replay<Dual> R = replay<Dual>(cx, path, p, d, L[i], first_photon_id + i, key, tr, delta);
                        if (!R.ok) break;
                        Dual m;
                        if (objective == 1 && !exit_margin<Dual>(scene, v, R.p, R.d, &m)) break;
                        for (int j = 0; j < tr.n; ++j) {
                            const o_surface& ts = scene->surfaces[tr.sid[j]];
                            const int base = ts.shape == O_SHAPE_SAG ? 0 : 10;
                            const int nslots = ts.shape == O_SHAPE_SAG ? 10 : 6;
                            for (int k2 = 0; k2 < nslots; ++k2) {
                                const int sl = 10 * j + k2;
                                double c;
                                if (centroid) {
                                    c = w[i] / Wv[v] * (cax == 0 ? R.qx.d[sl] : R.qy.d[sl]);
                                } else if (objective == 0) {
                                    c = 2.0 * w[i] / Wv[v] *
                                        ((qx[i] - cxv[v]) * R.qx.d[sl] + (qy[i] - cyv[v]) * R.qy.d[sl]);
                                } else {
                                    const double sg = sigmoid(m.v / tau);
                                    c = w[i] * sg * (1.0 - sg) / tau * m.d[sl] / nv[v];
                                }
                                g[(size_t)tr.sid[j] * O_N_PARAM + base + k2] += c;
                            }
                        }
                    }
                }
            });
        for (auto& t : th) t.join();
    }
    std::fill(grad, grad + NP, 0.0);
    for (int k = 0; k < n_threads; ++k)
        for (size_t j = 0; j < NP; ++j) grad[j] += part[k][j];
    return 0;
}

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    philox(ctr, key, out);
}

int64_t oracle_track(const o_scene* scene, int64_t n, const double* O, const double* D, const double* L,
                     const int32_t* vop, uint64_t seed, int64_t first_photon_id, int32_t max_bounces, double eps,
                     int64_t track_first, int64_t track_count, double* points, int32_t* info, int64_t cap) {
    if (check_scene(scene) || n <= 0 || track_first < 0 || track_count < 0 || track_first + track_count > n) return -1;
    Ctx cx;
    cx.sc = scene;
    cx.frames.resize(scene->n_surfaces);
    for (int s = 0; s < scene->n_surfaces; ++s) cx.frames[s] = make_frame(scene->surfaces[s]);
    cx.eps = eps;
    cx.newton_tol = eps * 1e-4;
    std::vector<uint8_t> st(n), nb(n);
    o_outputs out{};
    out.status = st.data();
    out.bounces = nb.data();
    std::vector<TrackRec> recs;
    trace_range(cx, track_first, track_first + track_count, n, O, D, L, vop, seed, first_photon_id, max_bounces, &out,
                &recs);
    for (size_t k = 0; k < recs.size() && (int64_t)k < cap; ++k) {
        points[3 * k + 0] = recs[k].p.x;
        points[3 * k + 1] = recs[k].p.y;
        points[3 * k + 2] = recs[k].p.z;
        info[4 * k + 0] = (int32_t)recs[k].photon;
        info[4 * k + 1] = recs[k].bounce;
        info[4 * k + 2] = recs[k].sid;
        info[4 * k + 3] = recs[k].status;
    }
    return (int64_t)recs.size();
}

double oracle_fresnel_unpolarised(double n1, double n2, double cos_i) { return fresnel(n1, n2, cos_i); }
double oracle_refractive_index(const o_medium* m, double lambda_nm) { return refr_index(*m, lambda_nm); }
double oracle_absorption_length(const o_medium* m, double lambda_nm) { return abs_length(*m, lambda_nm); }
double oracle_reflectivity(const o_material* m, double lambda_nm) { return reflectivity(*m, lambda_nm); }

int oracle_intersect(const o_surface* s, const double p[3], const double d[3], double eps, double* t,
                     double n_front[3], double local_hit[3]) {
    Frame f = make_frame(*s);
    LocalHit lh;
    std::vector<Cand> cands;
    bool ok = intersect_surface(*s, f, v3(p[0], p[1], p[2]), v3(d[0], d[1], d[2]), eps, 1e-13, &lh, &cands);
    if (!ok) return lh.error ? -1 : 0;
    V3 nw = to_world_vec(f, lh.nl);
    *t = lh.t;
    n_front[0] = nw.x;
    n_front[1] = nw.y;
    n_front[2] = nw.z;
    local_hit[0] = lh.pl.x;
    local_hit[1] = lh.pl.y;
    local_hit[2] = lh.pl.z;
    return 1;
}

int oracle_trace(const o_scene* scene, int64_t n, const double* origins, const double* dirs,
                 const double* wavelengths, const int32_t* variant_of_photon, uint64_t seed,
                 int64_t first_photon_id, int32_t max_bounces, double eps, int32_t n_threads,
                 const o_outputs* out) {
    int rc = check_scene(scene);
    if (rc) return rc;
    if (n < 0 || max_bounces <= 0 || max_bounces > 255 || !out || !out->status || !out->bounces) return -10;
    if (n == 0) return 0;
    Ctx cx;
    cx.sc = scene;
    cx.frames.resize(scene->n_surfaces);
    for (int s = 0; s < scene->n_surfaces; ++s) cx.frames[s] = make_frame(scene->surfaces[s]);
    cx.eps = eps;
    cx.newton_tol = eps * 1e-4;
    if (n_threads <= 0) n_threads = 1;
    if ((int64_t)n_threads > n) n_threads = (int32_t)n;
    std::vector<std::thread> th;
    for (int k = 0; k < n_threads; ++k) {
        int64_t i0 = n * k / n_threads, i1 = n * (k + 1) / n_threads;
        th.emplace_back(trace_range, std::cref(cx), i0, i1, n, origins, dirs, wavelengths, variant_of_photon,
                        seed, first_photon_id, max_bounces, out, (std::vector<TrackRec>*)nullptr);
    }
    for (auto& t : th) t.join();
    return 0;
}

}  // extern "C"
