/*
 * pt_oracle.c -- CPU oracle for the path tracer. TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, recursive Monte Carlo path tracer in double precision.  It is the
 * reference that the CUDA path is checked against and it shares no code with it:
 * only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs
 * may load it.
 *
 * What it computes (paper: "Physically-based Path Tracer using WebGPU and OpenPBR"):
 *   - the pixel estimate of the rendering equation I = g [eps + int p I]   (Sec. 1.1, Eq. 1)
 *     by backward path tracing from a perspective camera with per-sample jitter (Sec. 5.1.2),
 *   - closest-hit search through an AABB BVH (Sec. 5.1.1); a brute-force loop over all
 *     triangles is kept beside it as the pin,
 *   - OpenPBR-style shading at every hit with importance sampling (Sec. 4, Sec. 5.1.3),
 *   - Russian roulette and averaging of the samples (Sec. 5.1.3), progressive (Sec. 5.1.4),
 *   - optionally ReSTIR DI at the primary vertex (the paper's pointer to reservoir
 *     resampling for many lights, Sec. 2 and Sec. 6.3; Bitterli et al. 2020), as passes
 *     over the window per sample index.
 * Where the paper is silent (light sampling, MIS, the RNG keying, the lobe formulas, camera
 * conventions, depth semantics, roulette rule) this file follows the readings listed in the
 * design notes; each such place says "reading:" below.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), counter
 * (pixel, sample, bounce, dim/4), key (lo32(seed), hi32(seed)), word dim%4, uniform
 * U = (word >> 8) * 2^-24.  Reading: the paper uses PCG (Sec. 5.1.2); a counter-based
 * generator is used instead so the oracle and the GPU draw identical numbers.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------------------ */
/* small vector algebra                                                                   */
/* ------------------------------------------------------------------------------------ */
typedef struct { double x, y, z; } v3;

static inline v3 mk(double x, double y, double z) { v3 r; r.x = x; r.y = y; r.z = z; return r; }
static inline v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static inline v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static inline v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static inline v3 hmul(v3 a, v3 b) { return mk(a.x * b.x, a.y * b.y, a.z * b.z); }
static inline double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static inline v3 cross(v3 a, v3 b) {
    return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static inline double length(v3 a) { return sqrt(dot(a, a)); }
static inline v3 normalize(v3 a) { return scl(a, 1.0 / length(a)); }
static inline double get(v3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }
static inline double lum(v3 c) { return 0.2126 * c.x + 0.7152 * c.y + 0.0722 * c.z; }
static inline double maxc(v3 c) { return fmax(c.x, fmax(c.y, c.z)); }
static inline v3 splat(double s) { return mk(s, s, s); }

/* ------------------------------------------------------------------------------------ */
/* Philox4x32-10                                                                          */
/* ------------------------------------------------------------------------------------ */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod_a = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t prod_b = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(prod_b >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)prod_b;
        uint32_t y2 = (uint32_t)(prod_a >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)prod_a;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;  /* Weyl key schedule */
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

double oracle_uniform(uint32_t pixel, uint32_t sample, uint32_t bounce, uint32_t dim,
                      uint64_t seed) {
    uint32_t ctr[4] = {pixel, sample, bounce, dim >> 2};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    return (double)(out[dim & 3u] >> 8) * (1.0 / 16777216.0);
}

/* dimension table of one path vertex */
enum { DIM_CAM_X = 0, DIM_CAM_Y = 1, DIM_LIGHT_PICK = 2, DIM_LIGHT_U = 3, DIM_LIGHT_V = 4,
       DIM_LOBE = 5, DIM_DIR_U = 6, DIM_DIR_V = 7, DIM_REFRACT = 8, DIM_RR = 9,
       DIM_LENS_U = 12, DIM_LENS_V = 13 };

/* ------------------------------------------------------------------------------------ */
/* OpenPBR parameters (OPBR_N = 34 values per material, same order as the C-ABI table)   */
/* ------------------------------------------------------------------------------------ */
#define OPBR_N 34
typedef struct {
    double base_weight; v3 base_color; double metalness; double diffuse_roughness;
    double spec_weight; v3 spec_color; double spec_rough; double spec_ior;
    double trans_weight; v3 trans_color;
    double coat_weight; v3 coat_color; double coat_rough; double coat_ior;
    double emission; v3 emission_color;
    int thin_walled;
    double spec_aniso;    /* specular_roughness_anisotropy in [0, 1] */
    double spec_rot;      /* tangent rotation about the normal, in turns */
    double fuzz_weight; v3 fuzz_color; double fuzz_rough;
} omat;

static omat unpack_material(const double* p) {
    omat m;
    m.base_weight = p[0]; m.base_color = mk(p[1], p[2], p[3]);
    m.metalness = p[4]; m.diffuse_roughness = p[5];
    m.spec_weight = p[6]; m.spec_color = mk(p[7], p[8], p[9]);
    m.spec_rough = p[10]; m.spec_ior = p[11];
    m.trans_weight = p[12]; m.trans_color = mk(p[13], p[14], p[15]);
    m.coat_weight = p[16]; m.coat_color = mk(p[17], p[18], p[19]);
    m.coat_rough = p[20]; m.coat_ior = p[21];
    m.emission = p[22]; m.emission_color = mk(p[23], p[24], p[25]);
    m.thin_walled = p[26] != 0.0;
    m.spec_aniso = p[27]; m.spec_rot = p[28];
    m.fuzz_weight = p[29]; m.fuzz_color = mk(p[30], p[31], p[32]); m.fuzz_rough = p[33];
    return m;
}

/* ------------------------------------------------------------------------------------ */
/* Fresnel                                                                                */
/* ------------------------------------------------------------------------------------ */
/* Exact unpolarised dielectric Fresnel reflectance.  cos_i = cosine on the incident side
 * (clamped to [0, 1]); eta = n_transmitted / n_incident.  Total internal reflection -> 1. */
double oracle_fresnel_dielectric(double cos_i, double eta) {
    if (cos_i < 0.0) cos_i = 0.0;
    if (cos_i > 1.0) cos_i = 1.0;
    double sin2_t = (1.0 - cos_i * cos_i) / (eta * eta);
    if (sin2_t >= 1.0) return 1.0;
    double cos_t = sqrt(1.0 - sin2_t);
    double r_par = (eta * cos_i - cos_t) / (eta * cos_i + cos_t);
    double r_perp = (cos_i - eta * cos_t) / (cos_i + eta * cos_t);
    return 0.5 * (r_par * r_par + r_perp * r_perp);
}

/* Metal Fresnel: Schlick's curve from F0, corrected by a mu(1-mu)^6 term so that at the
 * 82-degree reference angle (mu = 1/7) it equals tint * Schlick (the "F82-tint" model of the
 * Adobe Standard Material that OpenPBR adopts).  Clamped to [0, 1].
 * Reading: OpenPBR's metal Fresnel; base_weight*base_color is F0, specular_color the tint. */
static double f82_channel(double f0, double tint, double mu) {
    const double mu_bar = 1.0 / 7.0;
    double one_m = 1.0 - mu;
    double schlick = f0 + (1.0 - f0) * pow(one_m, 5.0);
    double schlick_bar = f0 + (1.0 - f0) * pow(1.0 - mu_bar, 5.0);
    double b = schlick_bar * (1.0 - tint) / (mu_bar * pow(1.0 - mu_bar, 6.0));
    double f = schlick - b * mu * pow(one_m, 6.0);
    return f < 0.0 ? 0.0 : (f > 1.0 ? 1.0 : f);
}
static v3 fresnel_f82(v3 f0, v3 tint, double mu) {
    if (mu < 0.0) mu = 0.0;
    if (mu > 1.0) mu = 1.0;
    return mk(f82_channel(f0.x, tint.x, mu), f82_channel(f0.y, tint.y, mu),
              f82_channel(f0.z, tint.z, mu));
}
void oracle_fresnel_f82(const double f0[3], const double tint[3], double mu, double out[3]) {
    v3 r = fresnel_f82(mk(f0[0], f0[1], f0[2]), mk(tint[0], tint[1], tint[2]), mu);
    out[0] = r.x; out[1] = r.y; out[2] = r.z;
}

/* ------------------------------------------------------------------------------------ */
/* GGX microfacet distribution (Trowbridge-Reitz), anisotropic: ax is the width along the */
/* tangent (local x), ay along the bitangent (local y); ax = ay = roughness^2 is isotropic. */
/* ------------------------------------------------------------------------------------ */
double oracle_ggx_D(const double h[3], double ax, double ay) {
    if (h[2] <= 0.0) return 0.0;
    double x = h[0] / ax, y = h[1] / ay;
    double d = x * x + y * y + h[2] * h[2];
    return 1.0 / (M_PI * ax * ay * d * d);
}
static double ggx_D(v3 h, double ax, double ay) { double hh[3] = {h.x, h.y, h.z}; return oracle_ggx_D(hh, ax, ay); }

/* Smith Lambda for GGX: (-1 + sqrt(1 + a(w)^2 tan^2))/2 with a(w)^2 tan^2 =
 * (ax^2 wx^2 + ay^2 wy^2) / wz^2, written without cancellation. */
static double ggx_lambda(v3 w, double ax, double ay) {
    double c2 = w.z * w.z;
    if (c2 <= 0.0) return INFINITY;
    double x = (ax * ax * w.x * w.x + ay * ay * w.y * w.y) / c2;
    return x / (2.0 * (1.0 + sqrt(1.0 + x)));
}
double oracle_ggx_G1(const double w[3], double ax, double ay) {
    return 1.0 / (1.0 + ggx_lambda(mk(w[0], w[1], w[2]), ax, ay));
}
static double ggx_G1(v3 w, double ax, double ay) { return 1.0 / (1.0 + ggx_lambda(w, ax, ay)); }
/* height-correlated masking-shadowing */
static double ggx_G2(v3 wo, v3 wi, double ax, double ay) {
    return 1.0 / (1.0 + ggx_lambda(wo, ax, ay) + ggx_lambda(wi, ax, ay));
}
/* density of visible normals: G1(wo) max(0, wo.h) D(h) / wo.z */
static double ggx_vndf_pdf(v3 wo, v3 h, double ax, double ay) {
    double oh = dot(wo, h);
    if (oh <= 0.0 || wo.z <= 0.0) return 0.0;
    return ggx_G1(wo, ax, ay) * oh * ggx_D(h, ax, ay) / wo.z;
}
/* Sampling of visible normals (Heitz, JCGT 7(4), 2018): stretch the view vector to the
 * unit-roughness configuration, sample the projected hemisphere, unstretch. */
static v3 ggx_vndf_sample(v3 wo, double ax, double ay, double u1, double u2) {
    v3 vh = normalize(mk(ax * wo.x, ay * wo.y, wo.z));
    double lensq = vh.x * vh.x + vh.y * vh.y;
    v3 t1 = lensq > 0.0 ? scl(mk(-vh.y, vh.x, 0.0), 1.0 / sqrt(lensq)) : mk(1.0, 0.0, 0.0);
    v3 t2 = cross(vh, t1);
    double r = sqrt(u1);
    double phi = 2.0 * M_PI * u2;
    double p1 = r * cos(phi);
    double p2 = r * sin(phi);
    double s = 0.5 * (1.0 + vh.z);
    p2 = (1.0 - s) * sqrt(fmax(0.0, 1.0 - p1 * p1)) + s * p2;
    v3 nh = add(add(scl(t1, p1), scl(t2, p2)), scl(vh, sqrt(fmax(0.0, 1.0 - p1 * p1 - p2 * p2))));
    return normalize(mk(ax * nh.x, ay * nh.y, fmax(0.0, nh.z)));
}
void oracle_ggx_vndf_sample(const double wo[3], double ax, double ay, double u1, double u2, double out[3]) {
    v3 h = ggx_vndf_sample(mk(wo[0], wo[1], wo[2]), ax, ay, u1, u2);
    out[0] = h.x; out[1] = h.y; out[2] = h.z;
}

/* ------------------------------------------------------------------------------------ */
/* Fuzz lobe (OpenPBR fuzz layer; reading).  A microfacet sheen lobe: the "Charlie"       */
/* distribution of Estevez & Kulla 2017, D(m) = (2 + 1/a) sin(theta_m)^(1/a) / (2 pi) with  */
/* a = max(fuzz_roughness, 0.2)^2, and its exact Smith masking.  The masking of a          */
/* distribution follows from its projected area A(mu) = int <w, m>+ D(m) dm (G1 = mu / A,  */
/* Lambda = A / mu - 1; Heitz 2014), so the height-correlated lobe is                     */
/*   f_s(wo, wi) = D(h) G2 / (4 mu_i mu_o) = D(h) / (4 (A(mu_i) mu_o + A(mu_o) mu_i - mu_i mu_o)). */
/* A has no closed form for this D: it and the lobe's directional albedo                   */
/*   E(mu_o) = int f_s(wo, wi) mu_i dwi                                                   */
/* are integrated numerically below, every time they are needed (Gauss-Legendre rules).  */
/* ------------------------------------------------------------------------------------ */
#define GL_N 64
#define GL_M 24   /* points per polar piece of the albedo rule */
static double gl_x[GL_N], gl_w[GL_N];   /* Gauss-Legendre nodes and weights on [-1, 1] */
static double glm_x[GL_M], glm_w[GL_M];
static pthread_once_t gl_once = PTHREAD_ONCE_INIT;

/* nodes = roots of the Legendre polynomial P_n, by Newton's method from the usual
 * cos(pi (j + 3/4) / (n + 1/2)) guesses; weights 2 / ((1 - x^2) P_n'(x)^2) */
static void gl_rule(int n, double* xs, double* ws) {
    for (int j = 0; j < n; ++j) {
        double x = cos(M_PI * (j + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        xs[j] = x;
        ws[j] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

static void gl_init(void) {
    gl_rule(GL_N, gl_x, gl_w);
    gl_rule(GL_M, glm_x, glm_w);
}

/* node j of the 64-point rule mapped to [a, b], with its weight */
static void gl_node(double a, double b, int j, double* t, double* w) {
    pthread_once(&gl_once, gl_init);
    *t = 0.5 * (b + a) + 0.5 * (b - a) * gl_x[j];
    *w = 0.5 * (b - a) * gl_w[j];
}

static double fuzz_alpha(double rough) {
    double r = fmax(rough, 0.2);
    return r * r;
}

/* Charlie distribution at a microfacet normal with cosine cos_m to the surface normal */
double oracle_sheen_D(double cos_m, double alpha) {
    double s2 = fmax(0.0, 1.0 - cos_m * cos_m);
    return (2.0 + 1.0 / alpha) * pow(s2, 0.5 / alpha) / (2.0 * M_PI);
}

/* A(mu) = int D(theta_m) sin(theta_m) int_0^{2pi} max(0, a cos(phi) + b) dphi dtheta_m with
 * a = sin(theta) sin(theta_m), b = mu cos(theta_m).  The inner integral is 2 pi b where
 * b >= a (theta_m <= asin(mu): the whole circle faces w) and 2 a sin(phi0) + 2 b phi0 with
 * cos(phi0) = -b/a elsewhere; the theta_m integral is split at that kink. */
double oracle_sheen_area(double mu, double alpha) {
    mu = fmin(fmax(mu, 0.0), 1.0);
    const double st = sqrt(fmax(0.0, 1.0 - mu * mu)), split = asin(mu);
    double sum = 0.0;
    for (int j = 0; j < GL_N; ++j) {
        double th, w;
        gl_node(0.0, split, j, &th, &w);
        sum += w * oracle_sheen_D(cos(th), alpha) * sin(th) * 2.0 * M_PI * mu * cos(th);
    }
    for (int j = 0; j < GL_N; ++j) {
        double th, w;
        gl_node(split, 0.5 * M_PI, j, &th, &w);
        const double a = st * sin(th), b = mu * cos(th);
        double inner;
        if (b >= a) {
            inner = 2.0 * M_PI * b;
        } else {
            const double c = -b / a;
            inner = 2.0 * a * sqrt(fmax(0.0, 1.0 - c * c)) + 2.0 * b * acos(c);
        }
        sum += w * oracle_sheen_D(cos(th), alpha) * sin(th) * inner;
    }
    return sum;
}

/* the sheen lobe for wo, wi above the surface, given A at both cosines */
static double sheen_f(v3 wo, v3 wi, double alpha, double a_o, double a_i) {
    v3 h = normalize(add(wo, wi));
    return oracle_sheen_D(h.z, alpha) / (4.0 * (a_i * wo.z + a_o * wi.z - wi.z * wo.z));
}

double oracle_sheen_f(const double wo[3], const double wi[3], double alpha) {
    if (wo[2] <= 0.0 || wi[2] <= 0.0) return 0.0;
    return sheen_f(mk(wo[0], wo[1], wo[2]), mk(wi[0], wi[1], wi[2]), alpha, oracle_sheen_area(wo[2], alpha),
                   oracle_sheen_area(wi[2], alpha));
}

/* E(mu_o) = int f_s(wo, wi) mu_i dwi with wo = (sin, 0, mu_o).  The integrand is even in the
 * azimuth of wi, so E = 2 int sin(th_i) cos(th_i) dth_i int_0^pi dphi f_s.  The lobe turns over
 * where mu_i ~ mu_o and has a kink at the mirror direction (mu_i = mu_o, phi = pi), so the polar
 * range is cut at mu_i = c, 4 c, 16 c, ... up to 1 with c = max(mu_o, 1e-6) (the floor keeps the
 * features at the horizon resolved for a horizontal wo; the piece below 1e-6 holds at most
 * about 1e-6 of E); each piece is integrated over the polar angle (smooth through the pole,
 * where mu_i is not) with 24 points.  In a piece whose mu_i stays below mu_hi the features
 * next to phi = pi are about mu_o + mu_hi wide, so its azimuth range is cut at
 * pi - min(pi, 8 (mu_o + mu_hi)), 64 points a part.  This rule agrees with adaptive quadrature
 * of the same lobe to about 1e-9 at every mu_o. */
double oracle_sheen_albedo(double mu_o, double alpha) {
    pthread_once(&gl_once, gl_init);
    mu_o = fmin(fmax(mu_o, 0.0), 1.0);
    const v3 wo = mk(sqrt(fmax(0.0, 1.0 - mu_o * mu_o)), 0.0, mu_o);
    const double a_o = oracle_sheen_area(mu_o, alpha);
    double sum = 0.0, lo = 0.0, hi = fmax(mu_o, 1e-6);
    while (lo < 1.0) {
        const double t0 = acos(hi), t1 = acos(lo);
        const double cut = fmin(M_PI, 8.0 * (mu_o + hi));
        for (int i = 0; i < GL_M; ++i) {
            const double th = 0.5 * (t0 + t1) + 0.5 * (t1 - t0) * glm_x[i];
            const double wt = 0.5 * (t1 - t0) * glm_w[i];
            const double mi = cos(th), si = sin(th);
            const double a_i = oracle_sheen_area(mi, alpha);
            for (int part = 0; part < 2; ++part) {
                const double p0 = part == 0 ? 0.0 : M_PI - cut, p1 = part == 0 ? M_PI - cut : M_PI;
                if (p1 <= p0) continue;
                for (int j = 0; j < GL_N; ++j) {
                    double ph, wp;
                    gl_node(p0, p1, j, &ph, &wp);
                    const v3 wi = mk(si * cos(ph), si * sin(ph), mi);
                    sum += wt * wp * sheen_f(wo, wi, alpha, a_o, a_i) * mi * si;
                }
            }
        }
        lo = hi;
        hi = fmin(4.0 * lo, 1.0);
    }
    return 2.0 * sum;
}

static v3 reflect(v3 wo, v3 h) { return sub(scl(h, 2.0 * dot(wo, h)), wo); }
/* refraction of wo (on the +h side) into the medium with relative index eta; 0 on TIR */
static int refract(v3 wo, v3 h, double eta, v3* wi) {
    double ci = dot(wo, h);
    double s2t = (1.0 - ci * ci) / (eta * eta);
    if (s2t >= 1.0) return 0;
    double ct = sqrt(1.0 - s2t);
    *wi = add(scl(wo, -1.0 / eta), scl(h, ci / eta - ct));
    return 1;
}

/* ------------------------------------------------------------------------------------ */
/* OpenPBR subset as a mixture of lobes (local frame, shading normal = +z, wo.z > 0)      */
/*                                                                                        */
/* Reading of the layering (OpenPBR is not fully specified in the paper, Sec. 4):          */
/*   f = cw f_coat + A_c (m f_metal + (1-m) f_diel)                                       */
/*   A_c(mi, mo) = cw cc (1 - Fc(|mi|)) (1 - Fc(mo)) + (1 - cw)                           */
/*   f_metal = sw F82(bw bc, sc, wo.h) D G2 / (4 mo mi)                                   */
/*   f_diel  = sw sc F(wo.h) D G2 / (4 mo mi)                                              */
/*           + (1-t) (1 - sw F(|mi|)) (1 - sw F(mo)) bw bc / pi                             */
/*           + t tc (1 - sw F(wo.h)) D G2 |wi.h| (wo.h) / (|mi| mo (wo.h + eta wi.h)^2)     */
/*   f_coat  = Fc(wo.h) Dc G2c / (4 mo mi)                                                 */
/* alpha < 1e-4 makes a lobe a delta lobe.  eta = specular_ior seen from the side of wo:   */
/* for transmissive materials hit from the back it is 1/ior.                             */
/* Thin-walled (reading of OpenPBR's geometry_thin_walled): both sides alike (eta = ior),  */
/* and the transmission term is the reflection microfacet lobe mirrored through the       */
/* surface plane: with wi' = (wi.x, wi.y, -wi.z) and h the half vector of (wo, wi'),       */
/*   f_t = t tc (1 - sw F(wo.h)) D G2(wo, wi') / (4 mo |mi|)   (no refraction, no 1/eta^2) */
/* Specular anisotropy (OpenPBR specular_roughness_anisotropy a): the specular GGX lobe of  */
/* metal, dielectric and transmission has widths ax = r^2 sqrt(2 / (1 + (1-a)^2)) along the */
/* tangent and ay = (1-a) ax along the bitangent, in the frame of tangent_frame (the coat  */
/* stays isotropic).                                                                      */
/* ------------------------------------------------------------------------------------ */
/* Fuzz (OpenPBR's fuzz layer over the coat; reading): with fuzz weight fw, colour fc,    */
/*   f = fw fc f_s + A_f (cw f_coat + A_c (...)),                                           */
/*   A_f(mu_i, mu_o) = (1 - fw) + fw (1 - E(|mu_i|)) (1 - E(mu_o)),                         */
/* E the sheen lobe's albedo (the light that the fibres do not send back passes them, on   */
/* the way in and on the way out; symmetric like the coat's factor).  The fuzz lobe is     */
/* sampled uniformly over the upper hemisphere (z = u1, phi = 2 pi u2), picked with weight */
/* fw lum(fc) E(mu_o); the other lobes' weights are scaled by 1 - fw E(mu_o).              */
enum { LOBE_COAT = 0, LOBE_METAL = 1, LOBE_DIEL = 2, LOBE_DIFF = 3, LOBE_FUZZ = 4, N_LOBES = 5 };

typedef struct {
    omat m;
    double eta_s, eta_c;
    double ax_s, ay_s, a_c;   /* specular widths along tangent / bitangent; coat (isotropic) */
    int delta_s, delta_c;
    double alpha_f, a_fo, e_fo;   /* fuzz: Charlie width, A(mu_o), E(mu_o) */
    double p[N_LOBES];     /* lobe selection probabilities */
    int any;               /* some lobe has positive weight */
    int has_smooth;        /* some non-delta lobe has positive weight */
} closure;

static void closure_setup(closure* C, const omat* m, int front, double mu_o) {
    C->m = *m;
    C->eta_s = (m->trans_weight > 0.0 && !front && !m->thin_walled) ? 1.0 / m->spec_ior : m->spec_ior;
    C->eta_c = m->coat_ior;
    /* OpenPBR's anisotropy mapping: the tangent width grows and the bitangent width shrinks
     * with a, keeping ax^2 + ay^2 = 2 r^4; a = 0 gives ax = ay = r^2.  The lobe is a delta
     * lobe when both widths are below 1e-4; otherwise the narrower one is kept >= 1e-4. */
    double r2 = m->spec_rough * m->spec_rough, ia = 1.0 - m->spec_aniso;
    double at = r2 * sqrt(2.0 / (1.0 + ia * ia));
    C->ax_s = at;
    C->ay_s = fmax(ia * at, 1e-4);
    C->a_c = m->coat_rough * m->coat_rough;
    C->delta_s = at < 1e-4;
    C->delta_c = C->a_c < 1e-4;
    double fc = oracle_fresnel_dielectric(mu_o, C->eta_c);
    double w_coat = m->coat_weight * fc;
    double att = m->coat_weight * lum(m->coat_color) * (1.0 - fc) + (1.0 - m->coat_weight);
    v3 f0 = scl(m->base_color, m->base_weight);
    double w_metal = att * m->metalness * m->spec_weight * lum(fresnel_f82(f0, m->spec_color, mu_o));
    double fs = oracle_fresnel_dielectric(mu_o, C->eta_s);
    double w_spec = att * (1.0 - m->metalness) * m->spec_weight * lum(m->spec_color) * fs;
    double w_trans = att * (1.0 - m->metalness) * m->trans_weight * lum(m->trans_color) *
                     (1.0 - m->spec_weight * fs);
    double w_diff = att * (1.0 - m->metalness) * (1.0 - m->trans_weight) *
                    (1.0 - m->spec_weight * fs) * lum(f0);
    double w[N_LOBES] = {w_coat, w_metal, w_spec + w_trans, w_diff, 0.0};
    C->alpha_f = fuzz_alpha(m->fuzz_rough);
    C->a_fo = C->e_fo = 0.0;
    if (m->fuzz_weight > 0.0) {
        C->a_fo = oracle_sheen_area(mu_o, C->alpha_f);
        C->e_fo = oracle_sheen_albedo(mu_o, C->alpha_f);
        for (int j = 0; j < LOBE_FUZZ; ++j) w[j] *= 1.0 - m->fuzz_weight * C->e_fo;
        w[LOBE_FUZZ] = m->fuzz_weight * lum(m->fuzz_color) * C->e_fo;
    }
    double sum = w[0] + w[1] + w[2] + w[3] + w[4];
    C->any = sum > 0.0;
    for (int j = 0; j < N_LOBES; ++j) C->p[j] = C->any ? w[j] / sum : 0.0;
    C->has_smooth = (C->p[LOBE_COAT] > 0.0 && !C->delta_c) ||
                    ((C->p[LOBE_METAL] > 0.0 || C->p[LOBE_DIEL] > 0.0) && !C->delta_s) ||
                    C->p[LOBE_DIFF] > 0.0 || C->p[LOBE_FUZZ] > 0.0;
}

/* A_f: how much of the layers under the fuzz reaches wo from wi (1 without fuzz) */
static double fuzz_attenuation(const closure* C, double mu_i_abs) {
    const omat* m = &C->m;
    if (!(m->fuzz_weight > 0.0)) return 1.0;
    double e_i = oracle_sheen_albedo(mu_i_abs, C->alpha_f);
    return (1.0 - m->fuzz_weight) + m->fuzz_weight * (1.0 - e_i) * (1.0 - C->e_fo);
}

/* probability of reflecting (vs refracting) in the dielectric lobe, given F(wo.h) */
static double diel_reflect_prob(const closure* C, double F) {
    const omat* m = &C->m;
    double r = m->spec_weight * lum(m->spec_color) * F;
    double t = m->trans_weight * lum(m->trans_color) * (1.0 - m->spec_weight * F);
    if (F >= 1.0) return 1.0;
    double s = r + t;
    return s > 0.0 ? r / s : 1.0;
}

static v3 coat_attenuation(const closure* C, double mu_i_abs, double mu_o) {
    const omat* m = &C->m;
    double fci = oracle_fresnel_dielectric(mu_i_abs, C->eta_c);
    double fco = oracle_fresnel_dielectric(mu_o, C->eta_c);
    return add(scl(m->coat_color, m->coat_weight * (1.0 - fci) * (1.0 - fco)),
               splat(1.0 - m->coat_weight));
}

/* non-delta part of f(wo, wi) and the mixture pdf of producing wi by BSDF sampling */
/* Rough diffuse (reading; the paper names OpenPBR, whose base_diffuse_roughness uses the
 * energy-preserving Oren-Nayar model): its single-scattering part, Fujii's qualitative
 * Oren-Nayar form, as a factor on the Lambert term:
 *   (1 + sigma * s / t) / (1 + c * sigma),  c = 1/2 - 2/(3 pi),
 *   s = wi.wo - mu_i mu_o,  t = max(mu_i, mu_o) if s > 0, else 1.
 * sigma = 0 is Lambert; the factor is symmetric in (wi, wo); the multiple-scattering
 * compensation is not included, so a rough diffuse surface loses a little energy. */
static double fon_factor(v3 wo, v3 wi, double sigma) {
    if (sigma <= 0.0) return 1.0;
    double s = dot(wo, wi) - wo.z * wi.z;
    double t = s > 0.0 ? fmax(wo.z, wi.z) : 1.0;
    return (1.0 + sigma * s / t) / (1.0 + (0.5 - 2.0 / (3.0 * M_PI)) * sigma);
}

static void closure_eval(const closure* C, v3 wo, v3 wi, v3* f_out, double* pdf_out) {
    const omat* m = &C->m;
    v3 f = splat(0.0);
    double pdf = 0.0;
    double mo = wo.z, mi = wi.z;
    *f_out = f;
    *pdf_out = 0.0;
    if (mo <= 0.0 || mi == 0.0) return;
    v3 ac = coat_attenuation(C, fabs(mi), mo);
    if (mi > 0.0) {
        v3 h = normalize(add(wo, wi));
        double oh = dot(wo, h);
        if (oh <= 0.0) return;
        if (!C->delta_c && m->coat_weight > 0.0) {
            double fr = oracle_fresnel_dielectric(oh, C->eta_c);
            double val = m->coat_weight * fr * ggx_D(h, C->a_c, C->a_c) * ggx_G2(wo, wi, C->a_c, C->a_c) /
                         (4.0 * mo * mi);
            f = add(f, splat(val));
            pdf += C->p[LOBE_COAT] * ggx_vndf_pdf(wo, h, C->a_c, C->a_c) / (4.0 * oh);
        }
        if (!C->delta_s) {
            double dg = ggx_D(h, C->ax_s, C->ay_s) * ggx_G2(wo, wi, C->ax_s, C->ay_s) / (4.0 * mo * mi);
            double vndf = ggx_vndf_pdf(wo, h, C->ax_s, C->ay_s) / (4.0 * oh);
            if (m->metalness > 0.0) {
                v3 fm = fresnel_f82(scl(m->base_color, m->base_weight), m->spec_color, oh);
                f = add(f, scl(hmul(ac, fm), m->metalness * m->spec_weight * dg));
            }
            pdf += C->p[LOBE_METAL] * vndf;
            double fr = oracle_fresnel_dielectric(oh, C->eta_s);
            f = add(f, scl(hmul(ac, m->spec_color), (1.0 - m->metalness) * m->spec_weight * fr * dg));
            pdf += C->p[LOBE_DIEL] * diel_reflect_prob(C, fr) * vndf;
        }
        double fsi = oracle_fresnel_dielectric(mi, C->eta_s);
        double fso = oracle_fresnel_dielectric(mo, C->eta_s);
        double kd = (1.0 - m->metalness) * (1.0 - m->trans_weight) * (1.0 - m->spec_weight * fsi) *
                    (1.0 - m->spec_weight * fso) * m->base_weight / M_PI * fon_factor(wo, wi, m->diffuse_roughness);
        f = add(f, scl(hmul(ac, m->base_color), kd));
        pdf += C->p[LOBE_DIFF] * mi / M_PI;
    } else if (m->thin_walled) {
        if (!C->delta_s && m->trans_weight > 0.0) {
            v3 wm = mk(wi.x, wi.y, -wi.z);
            v3 h = normalize(add(wo, wm));
            double oh = dot(wo, h);
            if (oh > 0.0) {
                double fr = oracle_fresnel_dielectric(oh, C->eta_s);
                double dg = ggx_D(h, C->ax_s, C->ay_s) * ggx_G2(wo, wm, C->ax_s, C->ay_s) / (4.0 * mo * fabs(mi));
                double val = (1.0 - m->metalness) * m->trans_weight * (1.0 - m->spec_weight * fr) * dg;
                f = add(f, scl(hmul(ac, m->trans_color), val));
                pdf += C->p[LOBE_DIEL] * (1.0 - diel_reflect_prob(C, fr)) * ggx_vndf_pdf(wo, h, C->ax_s, C->ay_s) /
                       (4.0 * oh);
            }
        }
    } else {
        if (!C->delta_s && m->trans_weight > 0.0) {
            double eta = C->eta_s;
            v3 h = normalize(add(wo, scl(wi, eta)));
            if (h.z < 0.0) h = scl(h, -1.0);
            double oh = dot(wo, h), ih = dot(wi, h);
            if (oh > 0.0 && ih < 0.0) {
                double fr = oracle_fresnel_dielectric(oh, eta);
                double denom = oh + eta * ih;
                double dg = ggx_D(h, C->ax_s, C->ay_s) * ggx_G2(wo, wi, C->ax_s, C->ay_s);
                double val = (1.0 - m->metalness) * m->trans_weight * (1.0 - m->spec_weight * fr) *
                             dg * fabs(ih) * oh / (fabs(mi) * mo * denom * denom);
                f = add(f, scl(hmul(ac, m->trans_color), val));
                pdf += C->p[LOBE_DIEL] * (1.0 - diel_reflect_prob(C, fr)) *
                       ggx_vndf_pdf(wo, h, C->ax_s, C->ay_s) * eta * eta * fabs(ih) / (denom * denom);
            }
        }
    }
    if (m->fuzz_weight > 0.0) {
        f = scl(f, fuzz_attenuation(C, fabs(mi)));
        if (mi > 0.0) {
            double fs = sheen_f(wo, wi, C->alpha_f, C->a_fo, oracle_sheen_area(mi, C->alpha_f));
            f = add(f, scl(m->fuzz_color, m->fuzz_weight * fs));
            pdf += C->p[LOBE_FUZZ] / (2.0 * M_PI);
        }
    }
    *f_out = f;
    *pdf_out = pdf;
}

typedef struct {
    v3 wi;
    v3 weight;     /* f |cos| / pdf (delta lobes: reflectance / selection probability) */
    double pdf;    /* mixture pdf of the non-delta lobes at wi (0 for a delta sample) */
    int is_delta;
} bsdf_sample_t;

/* one-sample mixture: pick a lobe with u_lobe, sample it with (u1, u2), dielectric
 * reflect/refract with u_refr.  Returns 0 if the sample is invalid (path ends). */
static int closure_sample(const closure* C, v3 wo, double u_lobe, double u1, double u2,
                          double u_refr, bsdf_sample_t* out) {
    const omat* m = &C->m;
    if (!C->any || wo.z <= 0.0) return 0;
    int lobe = -1, last = -1;
    double c = 0.0;
    for (int j = 0; j < N_LOBES; ++j) {
        if (C->p[j] <= 0.0) continue;
        last = j;
        c += C->p[j];
        if (u_lobe < c) { lobe = j; break; }
    }
    if (lobe < 0) lobe = last;
    double mo = wo.z;
    v3 wi;
    out->is_delta = 0;
    out->pdf = 0.0;
    if (lobe == LOBE_COAT) {
        if (C->delta_c) {
            out->wi = mk(-wo.x, -wo.y, wo.z);
            out->weight = splat(m->coat_weight * oracle_fresnel_dielectric(mo, C->eta_c) *
                                fuzz_attenuation(C, mo) / C->p[LOBE_COAT]);
            out->is_delta = 1;
            return 1;
        }
        v3 h = ggx_vndf_sample(wo, C->a_c, C->a_c, u1, u2);
        wi = reflect(wo, h);
        if (wi.z <= 0.0) return 0;
    } else if (lobe == LOBE_METAL) {
        if (C->delta_s) {
            out->wi = mk(-wo.x, -wo.y, wo.z);
            v3 fm = fresnel_f82(scl(m->base_color, m->base_weight), m->spec_color, mo);
            out->weight = scl(hmul(coat_attenuation(C, mo, mo), fm),
                              m->metalness * m->spec_weight * fuzz_attenuation(C, mo) / C->p[LOBE_METAL]);
            out->is_delta = 1;
            return 1;
        }
        v3 h = ggx_vndf_sample(wo, C->ax_s, C->ay_s, u1, u2);
        wi = reflect(wo, h);
        if (wi.z <= 0.0) return 0;
    } else if (lobe == LOBE_DIEL) {
        v3 h = C->delta_s ? mk(0.0, 0.0, 1.0) : ggx_vndf_sample(wo, C->ax_s, C->ay_s, u1, u2);
        double oh = dot(wo, h);
        if (oh <= 0.0) return 0;
        double fr = oracle_fresnel_dielectric(oh, C->eta_s);
        double pr = diel_reflect_prob(C, fr);
        int do_reflect = u_refr < pr;
        if (do_reflect) {
            wi = reflect(wo, h);
            if (wi.z <= 0.0) return 0;
        } else if (m->thin_walled) {
            /* the reflected direction mirrored through the surface plane */
            v3 wr = reflect(wo, h);
            if (wr.z <= 0.0) return 0;
            wi = mk(wr.x, wr.y, -wr.z);
        } else {
            if (!refract(wo, h, C->eta_s, &wi)) return 0;
            if (wi.z >= 0.0) return 0;
        }
        if (C->delta_s) {
            out->wi = wi;
            out->is_delta = 1;
            if (do_reflect) {
                out->weight = scl(hmul(coat_attenuation(C, mo, mo), m->spec_color),
                                  (1.0 - m->metalness) * m->spec_weight * fr * fuzz_attenuation(C, mo) /
                                      (C->p[LOBE_DIEL] * pr));
            } else {
                double scale = m->thin_walled ? 1.0 : C->eta_s * C->eta_s;   /* radiance across the interface */
                out->weight = scl(hmul(coat_attenuation(C, fabs(wi.z), mo), m->trans_color),
                                  (1.0 - m->metalness) * m->trans_weight *
                                      (1.0 - m->spec_weight * fr) * fuzz_attenuation(C, fabs(wi.z)) /
                                      (scale * C->p[LOBE_DIEL] * (1.0 - pr)));
            }
            return 1;
        }
    } else if (lobe == LOBE_DIFF) {
        double r = sqrt(u1), phi = 2.0 * M_PI * u2;
        wi = mk(r * cos(phi), r * sin(phi), sqrt(fmax(0.0, 1.0 - u1)));
        if (wi.z <= 0.0) return 0;
    } else {
        /* fuzz: uniform over the upper hemisphere */
        double r = sqrt(fmax(0.0, 1.0 - u1 * u1)), phi = 2.0 * M_PI * u2;
        wi = mk(r * cos(phi), r * sin(phi), u1);
        if (wi.z <= 0.0) return 0;
    }
    v3 f;
    double pdf;
    closure_eval(C, wo, wi, &f, &pdf);
    if (!(pdf > 0.0)) return 0;
    out->wi = wi;
    out->pdf = pdf;
    out->weight = scl(f, fabs(wi.z) / pdf);
    return 1;
}

/* ---- exported BSDF entry points (local frame) for the lobe pins and the GPU parity ---- */
void oracle_bsdf_eval(const double* matp, int front, const double wo[3], const double wi[3],
                      double f_out[3], double* pdf_out) {
    omat m = unpack_material(matp);
    closure C;
    closure_setup(&C, &m, front, wo[2]);
    v3 f;
    closure_eval(&C, mk(wo[0], wo[1], wo[2]), mk(wi[0], wi[1], wi[2]), &f, pdf_out);
    f_out[0] = f.x; f_out[1] = f.y; f_out[2] = f.z;
}

int oracle_bsdf_sample(const double* matp, int front, const double wo[3], const double u[4],
                       double wi_out[3], double weight_out[3], double* pdf_out, int* delta_out) {
    omat m = unpack_material(matp);
    closure C;
    closure_setup(&C, &m, front, wo[2]);
    bsdf_sample_t s;
    int ok = closure_sample(&C, mk(wo[0], wo[1], wo[2]), u[0], u[1], u[2], u[3], &s);
    if (!ok) { *pdf_out = 0.0; *delta_out = 0; return 0; }
    wi_out[0] = s.wi.x; wi_out[1] = s.wi.y; wi_out[2] = s.wi.z;
    weight_out[0] = s.weight.x; weight_out[1] = s.weight.y; weight_out[2] = s.weight.z;
    *pdf_out = s.pdf;
    *delta_out = s.is_delta;
    return 1;
}

void oracle_lobe_probs(const double* matp, int front, double mu_o, double out[5]) {
    omat m = unpack_material(matp);
    closure C;
    closure_setup(&C, &m, front, mu_o);
    for (int j = 0; j < N_LOBES; ++j) out[j] = C.p[j];
}

/* ------------------------------------------------------------------------------------ */
/* Scene                                                                                  */
/* ------------------------------------------------------------------------------------ */
typedef struct { double lo[3], hi[3]; int left, right, start, count; } bvh_node;

typedef struct {
    int n_mesh_tris, n_tris;       /* n_tris = mesh + 2 per quad light */
    v3* tv;                        /* 3 vertices per triangle */
    int* tri_mat;                  /* material id (mesh triangles) or -1-light index */
    int n_mats;
    omat* mats;
    int n_quads;
    v3 *q_p0, *q_e1, *q_e2, *q_L, *q_n;
    double* q_area;
    int* q_two_sided;
    int env_w, env_h;
    double* env;                   /* h * w * 3 */
    double* env_w_tex;             /* texel weights lum * sin(theta) */
    double* env_marg;              /* h + 1 */
    double* env_cond;              /* h * (w + 1) */
    double env_total;
    double eps;                    /* spawn offset */
    int use_bvh;
    bvh_node* nodes;
    int n_nodes;
    int* order;
} oscene;

/* ---- BVH: top-down median split on the longest centroid axis, leaves of <= 4 ---- */
typedef struct { double c[3]; double lo[3], hi[3]; int id; } prim_ref;

static void swap_ref(prim_ref* a, prim_ref* b) { prim_ref t = *a; *a = *b; *b = t; }

/* Hoare selection: puts the k-th smallest (by centroid on axis) at index k */
static void select_kth(prim_ref* r, int n, int k, int axis) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        double pivot = r[(lo + hi) / 2].c[axis];
        int i = lo, j = hi;
        while (i <= j) {
            while (r[i].c[axis] < pivot) ++i;
            while (r[j].c[axis] > pivot) --j;
            if (i <= j) { swap_ref(&r[i], &r[j]); ++i; --j; }
        }
        if (k <= j) hi = j;
        else if (k >= i) lo = i;
        else break;
    }
}

static int build_rec(oscene* S, prim_ref* r, int start, int count, int* next) {
    int ni = (*next)++;
    bvh_node* nd = &S->nodes[ni];
    double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int a = 0; a < 3; ++a) { nd->lo[a] = INFINITY; nd->hi[a] = -INFINITY; }
    for (int i = start; i < start + count; ++i)
        for (int a = 0; a < 3; ++a) {
            nd->lo[a] = fmin(nd->lo[a], r[i].lo[a]);
            nd->hi[a] = fmax(nd->hi[a], r[i].hi[a]);
            clo[a] = fmin(clo[a], r[i].c[a]);
            chi[a] = fmax(chi[a], r[i].c[a]);
        }
    if (count <= 4) {
        nd->left = nd->right = -1;
        nd->start = start;
        nd->count = count;
        return ni;
    }
    int axis = 0;
    for (int a = 1; a < 3; ++a)
        if (chi[a] - clo[a] > chi[axis] - clo[axis]) axis = a;
    int half = count / 2;
    select_kth(r + start, count, half, axis);
    nd->start = start;
    nd->count = 0;
    int l = build_rec(S, r, start, half, next);
    int rr = build_rec(S, r, start + half, count - half, next);
    S->nodes[ni].left = l;
    S->nodes[ni].right = rr;
    return ni;
}

static void build_bvh(oscene* S) {
    int n = S->n_tris;
    prim_ref* r = (prim_ref*)malloc(sizeof(prim_ref) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        v3 a = S->tv[3 * i], b = S->tv[3 * i + 1], c = S->tv[3 * i + 2];
        for (int ax = 0; ax < 3; ++ax) {
            double x = get(a, ax), y = get(b, ax), z = get(c, ax);
            r[i].lo[ax] = fmin(x, fmin(y, z));
            r[i].hi[ax] = fmax(x, fmax(y, z));
            r[i].c[ax] = (x + y + z) / 3.0;
        }
        r[i].id = i;
    }
    S->nodes = (bvh_node*)malloc(sizeof(bvh_node) * (size_t)(2 * (n > 0 ? n : 1)));
    int next = 0;
    if (n > 0) build_rec(S, r, 0, n, &next);
    S->n_nodes = next;
    S->order = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) S->order[i] = r[i].id;
    free(r);
}

/* ---- reference BVH quality: a binned surface-area-heuristic build ----
 * The quality of a BVH is judged here by the work a ray that enters the root box does on
 * average when it is tested against every box it meets (no early exit): with the probability
 * of meeting a box taken as its surface area over the root's (a uniform ray density, the
 * surface area heuristic of Goldsmith & Salmon, MacDonald & Booth),
 *   box tests = sum over internal nodes of A(node) / A(root) * (children of the node),
 *   triangle tests = sum over leaves of A(leaf) / A(root) * (triangles of the leaf).
 * The reference tree is binary, built top down: at each node 32 bins of the triangles'
 * centroids per axis, the split that minimises 2 + (A_L n_L + A_R n_R) / A (two child box
 * tests, then the triangles below, costed by the leaf estimate), a leaf when that is not
 * below n and n <= leaf_max.  It shares nothing with the device build (Morton codes, a radix
 * tree, an 8-wide collapse). */
static double box_area(const double lo[3], const double hi[3]) {
    double dx = fmax(hi[0] - lo[0], 0.0), dy = fmax(hi[1] - lo[1], 0.0), dz = fmax(hi[2] - lo[2], 0.0);
    return 2.0 * (dx * dy + dy * dz + dz * dx);
}

#define SAH_BINS 32
static void sah_rec(prim_ref* r, int count, int leaf_max, double root_area, double* box_tests, double* tri_tests,
                    int* n_nodes) {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = 0; i < count; ++i)
        for (int a = 0; a < 3; ++a) {
            lo[a] = fmin(lo[a], r[i].lo[a]);
            hi[a] = fmax(hi[a], r[i].hi[a]);
            clo[a] = fmin(clo[a], r[i].c[a]);
            chi[a] = fmax(chi[a], r[i].c[a]);
        }
    const double area = box_area(lo, hi);
    (*n_nodes)++;
    double best = INFINITY;
    int best_axis = -1, best_bin = -1;
    for (int a = 0; a < 3 && count > 1; ++a) {
        const double ext = chi[a] - clo[a];
        if (!(ext > 0.0)) continue;
        int bn[SAH_BINS] = {0};
        double blo[SAH_BINS][3], bhi[SAH_BINS][3];
        for (int b = 0; b < SAH_BINS; ++b)
            for (int k = 0; k < 3; ++k) { blo[b][k] = INFINITY; bhi[b][k] = -INFINITY; }
        for (int i = 0; i < count; ++i) {
            int b = (int)(SAH_BINS * (r[i].c[a] - clo[a]) / ext);
            if (b >= SAH_BINS) b = SAH_BINS - 1;
            bn[b]++;
            for (int k = 0; k < 3; ++k) {
                blo[b][k] = fmin(blo[b][k], r[i].lo[k]);
                bhi[b][k] = fmax(bhi[b][k], r[i].hi[k]);
            }
        }
        /* sweep: left areas and counts from the low side, right from the high side */
        double la[SAH_BINS], ra[SAH_BINS];
        int ln[SAH_BINS], rn[SAH_BINS];
        double l0[3] = {INFINITY, INFINITY, INFINITY}, l1[3] = {-INFINITY, -INFINITY, -INFINITY};
        int c = 0;
        for (int b = 0; b < SAH_BINS; ++b) {
            c += bn[b];
            for (int k = 0; k < 3; ++k) { l0[k] = fmin(l0[k], blo[b][k]); l1[k] = fmax(l1[k], bhi[b][k]); }
            ln[b] = c;
            la[b] = c ? box_area(l0, l1) : 0.0;
        }
        double r0[3] = {INFINITY, INFINITY, INFINITY}, r1[3] = {-INFINITY, -INFINITY, -INFINITY};
        c = 0;
        for (int b = SAH_BINS - 1; b >= 0; --b) {
            c += bn[b];
            for (int k = 0; k < 3; ++k) { r0[k] = fmin(r0[k], blo[b][k]); r1[k] = fmax(r1[k], bhi[b][k]); }
            rn[b] = c;
            ra[b] = c ? box_area(r0, r1) : 0.0;
        }
        for (int b = 0; b + 1 < SAH_BINS; ++b) {
            if (ln[b] == 0 || rn[b + 1] == 0) continue;
            const double cost = 2.0 + (la[b] * ln[b] + ra[b + 1] * rn[b + 1]) / area;
            if (cost < best) { best = cost; best_axis = a; best_bin = b; }
        }
    }
    if (count <= leaf_max && !(best < (double)count)) best_axis = -1;
    if (best_axis < 0 && count > leaf_max) {
        /* every centroid in one bin: split the list in halves */
        const int half = count / 2;
        *box_tests += 2.0 * area / root_area;
        sah_rec(r, half, leaf_max, root_area, box_tests, tri_tests, n_nodes);
        sah_rec(r + half, count - half, leaf_max, root_area, box_tests, tri_tests, n_nodes);
        return;
    }
    if (best_axis < 0) {
        *tri_tests += area / root_area * count;
        return;
    }
    const double ext = chi[best_axis] - clo[best_axis];
    int i = 0, j = count - 1;
    while (i <= j) {
        int b = (int)(SAH_BINS * (r[i].c[best_axis] - clo[best_axis]) / ext);
        if (b >= SAH_BINS) b = SAH_BINS - 1;
        if (b <= best_bin) ++i;
        else { swap_ref(&r[i], &r[j]); --j; }
    }
    *box_tests += 2.0 * area / root_area;
    sah_rec(r, i, leaf_max, root_area, box_tests, tri_tests, n_nodes);
    sah_rec(r + i, count - i, leaf_max, root_area, box_tests, tri_tests, n_nodes);
}

/* verts: n_tris * 9 doubles (three vertices per triangle); out: box tests, triangle tests,
 * nodes of the reference binned-SAH tree */
void oracle_sah_reference(const double* verts, int n_tris, int leaf_max, double* out) {
    out[0] = out[1] = out[2] = 0.0;
    if (n_tris <= 0) return;
    prim_ref* r = (prim_ref*)malloc(sizeof(prim_ref) * (size_t)n_tris);
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = 0; i < n_tris; ++i) {
        for (int ax = 0; ax < 3; ++ax) {
            double x = verts[9 * i + ax], y = verts[9 * i + 3 + ax], z = verts[9 * i + 6 + ax];
            r[i].lo[ax] = fmin(x, fmin(y, z));
            r[i].hi[ax] = fmax(x, fmax(y, z));
            r[i].c[ax] = (x + y + z) / 3.0;
            lo[ax] = fmin(lo[ax], r[i].lo[ax]);
            hi[ax] = fmax(hi[ax], r[i].hi[ax]);
        }
        r[i].id = i;
    }
    int nodes = 0;
    sah_rec(r, n_tris, leaf_max, box_area(lo, hi), &out[0], &out[1], &nodes);
    out[2] = nodes;
    free(r);
}

/* ---- environment map tables (reading: piecewise-constant 2D distribution over texels,
 *      weight = luminance * sin(theta at the texel centre)) ---- */
static void build_env(oscene* S) {
    int w = S->env_w, h = S->env_h;
    S->env_w_tex = (double*)malloc(sizeof(double) * (size_t)w * h);
    S->env_marg = (double*)malloc(sizeof(double) * (size_t)(h + 1));
    S->env_cond = (double*)malloc(sizeof(double) * (size_t)h * (w + 1));
    double total = 0.0;
    double* row = (double*)malloc(sizeof(double) * (size_t)h);
    for (int y = 0; y < h; ++y) {
        double st = sin(M_PI * (y + 0.5) / h);
        double rs = 0.0;
        for (int x = 0; x < w; ++x) {
            const double* t = &S->env[3 * ((size_t)y * w + x)];
            double wt = lum(mk(t[0], t[1], t[2])) * st;
            if (wt < 0.0) wt = 0.0;
            S->env_w_tex[(size_t)y * w + x] = wt;
            rs += wt;
        }
        row[y] = rs;
        double* cd = &S->env_cond[(size_t)y * (w + 1)];
        cd[0] = 0.0;
        double acc = 0.0;
        for (int x = 0; x < w; ++x) {
            acc += S->env_w_tex[(size_t)y * w + x];
            cd[x + 1] = rs > 0.0 ? acc / rs : (double)(x + 1) / w;
        }
        total += rs;
    }
    S->env_marg[0] = 0.0;
    double acc = 0.0;
    for (int y = 0; y < h; ++y) {
        acc += row[y];
        S->env_marg[y + 1] = total > 0.0 ? acc / total : (double)(y + 1) / h;
    }
    S->env_total = total;
    free(row);
}

void* oracle_scene_create(const double* vertices, int n_vertices, const uint32_t* indices,
                          int n_tris, const uint32_t* mat_ids, const double* mats, int n_mats,
                          const double* quads, int n_quads, const double* env, int env_w,
                          int env_h, int use_bvh) {
    (void)n_vertices;
    oscene* S = (oscene*)calloc(1, sizeof(oscene));
    S->n_mesh_tris = n_tris;
    S->n_tris = n_tris + 2 * n_quads;
    S->tv = (v3*)malloc(sizeof(v3) * 3 * (size_t)(S->n_tris > 0 ? S->n_tris : 1));
    S->tri_mat = (int*)malloc(sizeof(int) * (size_t)(S->n_tris > 0 ? S->n_tris : 1));
    for (int i = 0; i < n_tris; ++i) {
        for (int k = 0; k < 3; ++k) {
            const double* p = &vertices[3 * (size_t)indices[3 * (size_t)i + k]];
            S->tv[3 * i + k] = mk(p[0], p[1], p[2]);
        }
        S->tri_mat[i] = (int)mat_ids[i];
    }
    S->n_mats = n_mats;
    S->mats = (omat*)malloc(sizeof(omat) * (size_t)(n_mats > 0 ? n_mats : 1));
    for (int i = 0; i < n_mats; ++i) S->mats[i] = unpack_material(&mats[OPBR_N * i]);
    S->n_quads = n_quads;
    size_t nq = (size_t)(n_quads > 0 ? n_quads : 1);
    S->q_p0 = (v3*)malloc(sizeof(v3) * nq); S->q_e1 = (v3*)malloc(sizeof(v3) * nq);
    S->q_e2 = (v3*)malloc(sizeof(v3) * nq); S->q_L = (v3*)malloc(sizeof(v3) * nq);
    S->q_n = (v3*)malloc(sizeof(v3) * nq);
    S->q_area = (double*)malloc(sizeof(double) * nq);
    S->q_two_sided = (int*)malloc(sizeof(int) * nq);
    for (int l = 0; l < n_quads; ++l) {
        const double* q = &quads[13 * l];
        v3 p0 = mk(q[0], q[1], q[2]), e1 = mk(q[3], q[4], q[5]), e2 = mk(q[6], q[7], q[8]);
        S->q_p0[l] = p0; S->q_e1[l] = e1; S->q_e2[l] = e2;
        S->q_L[l] = mk(q[9], q[10], q[11]);
        v3 n = cross(e1, e2);
        S->q_area[l] = length(n);
        S->q_n[l] = normalize(n);
        S->q_two_sided[l] = q[12] != 0.0;
        /* the light is also geometry: two triangles appended after the mesh */
        int t0 = n_tris + 2 * l, t1 = t0 + 1;
        v3 p1 = add(p0, e1), p2 = add(add(p0, e1), e2), p3 = add(p0, e2);
        S->tv[3 * t0] = p0; S->tv[3 * t0 + 1] = p1; S->tv[3 * t0 + 2] = p2;
        S->tv[3 * t1] = p0; S->tv[3 * t1 + 1] = p2; S->tv[3 * t1 + 2] = p3;
        S->tri_mat[t0] = -1 - l;
        S->tri_mat[t1] = -1 - l;
    }
    S->env_w = env ? env_w : 0;
    S->env_h = env ? env_h : 0;
    if (env) {
        S->env = (double*)malloc(sizeof(double) * 3 * (size_t)env_w * env_h);
        memcpy(S->env, env, sizeof(double) * 3 * (size_t)env_w * env_h);
        build_env(S);
    }
    /* spawn offset: 1e-4 of the scene bounding-box diagonal (reading) */
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = 0; i < 3 * S->n_tris; ++i)
        for (int a = 0; a < 3; ++a) {
            lo[a] = fmin(lo[a], get(S->tv[i], a));
            hi[a] = fmax(hi[a], get(S->tv[i], a));
        }
    double diag = S->n_tris > 0 ? sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) +
                                       (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                                       (hi[2] - lo[2]) * (hi[2] - lo[2]))
                                : 1.0;
    S->eps = 1e-4 * diag;
    S->use_bvh = use_bvh;
    if (use_bvh) build_bvh(S);
    return S;
}

void oracle_scene_destroy(void* h) {
    oscene* S = (oscene*)h;
    if (!S) return;
    free(S->tv); free(S->tri_mat); free(S->mats);
    free(S->q_p0); free(S->q_e1); free(S->q_e2); free(S->q_L); free(S->q_n);
    free(S->q_area); free(S->q_two_sided);
    free(S->env); free(S->env_w_tex); free(S->env_marg); free(S->env_cond);
    free(S->nodes); free(S->order);
    free(S);
}

double oracle_scene_eps(void* h) { return ((oscene*)h)->eps; }

/* ------------------------------------------------------------------------------------ */
/* Ray / triangle: watertight test (Woop, Benthin, Wald, JCGT 2(1), 2013), in double      */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    v3 o, d;
    int kx, ky, kz;
    double sx, sy, sz;
} wray;

static wray make_wray(v3 o, v3 d) {
    wray r;
    r.o = o; r.d = d;
    double ad[3] = {fabs(d.x), fabs(d.y), fabs(d.z)};
    int kz = 0;
    if (ad[1] > ad[kz]) kz = 1;
    if (ad[2] > ad[kz]) kz = 2;
    int kx = (kz + 1) % 3, ky = (kx + 1) % 3;
    if (get(d, kz) < 0.0) { int t = kx; kx = ky; ky = t; }
    r.kx = kx; r.ky = ky; r.kz = kz;
    r.sx = get(d, kx) / get(d, kz);
    r.sy = get(d, ky) / get(d, kz);
    r.sz = 1.0 / get(d, kz);
    return r;
}

/* returns 1 and t (and barycentrics) if the ray hits the triangle with 0 < t < tmax */
static int tri_hit(const wray* r, v3 p0, v3 p1, v3 p2, double tmax, double* t_out,
                   double* u_out, double* v_out) {
    v3 A = sub(p0, r->o), B = sub(p1, r->o), C = sub(p2, r->o);
    double ax = get(A, r->kx) - r->sx * get(A, r->kz), ay = get(A, r->ky) - r->sy * get(A, r->kz);
    double bx = get(B, r->kx) - r->sx * get(B, r->kz), by = get(B, r->ky) - r->sy * get(B, r->kz);
    double cx = get(C, r->kx) - r->sx * get(C, r->kz), cy = get(C, r->ky) - r->sy * get(C, r->kz);
    double U = cx * by - cy * bx;
    double V = ax * cy - ay * cx;
    double W = bx * ay - by * ax;
    if ((U < 0.0 || V < 0.0 || W < 0.0) && (U > 0.0 || V > 0.0 || W > 0.0)) return 0;
    double det = U + V + W;
    if (det == 0.0) return 0;
    double az = r->sz * get(A, r->kz), bz = r->sz * get(B, r->kz), cz = r->sz * get(C, r->kz);
    double T = U * az + V * bz + W * cz;
    double t = T / det;
    if (!(t > 0.0) || !(t < tmax)) return 0;
    *t_out = t;
    *u_out = V / det;   /* weight of p1 */
    *v_out = W / det;   /* weight of p2 */
    return 1;
}

typedef struct { int tri; double t, u, v; } ohit;

static int box_hit(const bvh_node* n, v3 o, v3 d, double tmax, double* tnear_out) {
    double t0 = 0.0, t1 = tmax;
    for (int a = 0; a < 3; ++a) {
        double oa = get(o, a), da = get(d, a);
        if (da == 0.0) {
            if (oa < n->lo[a] || oa > n->hi[a]) return 0;
            continue;
        }
        double ta = (n->lo[a] - oa) / da, tb = (n->hi[a] - oa) / da;
        if (ta > tb) { double t = ta; ta = tb; tb = t; }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
    }
    /* slack keeps flat boxes (axis-aligned triangles) from being lost to rounding */
    if (t0 > t1 * (1.0 + 1e-9) + 1e-300) return 0;
    *tnear_out = t0;
    return 1;
}

static inline int closer(double t, int id, const ohit* best) {
    return t < best->t || (t == best->t && id < best->tri);
}

static void intersect_brute(const oscene* S, v3 o, v3 d, double tmax, ohit* h) {
    wray r = make_wray(o, d);
    h->tri = -1; h->t = tmax; h->u = h->v = 0.0;
    for (int i = 0; i < S->n_tris; ++i) {
        double t, u, v;
        if (tri_hit(&r, S->tv[3 * i], S->tv[3 * i + 1], S->tv[3 * i + 2], tmax, &t, &u, &v) &&
            (h->tri < 0 || closer(t, i, h))) {
            h->tri = i; h->t = t; h->u = u; h->v = v;
        }
    }
}

static void intersect_bvh(const oscene* S, v3 o, v3 d, double tmax, ohit* h) {
    wray r = make_wray(o, d);
    h->tri = -1; h->t = tmax; h->u = h->v = 0.0;
    if (S->n_tris == 0) return;
    int stack[128];
    int sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const bvh_node* n = &S->nodes[stack[--sp]];
        double tn;
        if (!box_hit(n, o, d, h->tri < 0 ? tmax : h->t, &tn)) continue;
        if (n->left < 0) {
            for (int k = n->start; k < n->start + n->count; ++k) {
                int i = S->order[k];
                double t, u, v;
                if (tri_hit(&r, S->tv[3 * i], S->tv[3 * i + 1], S->tv[3 * i + 2], tmax, &t, &u, &v) &&
                    (h->tri < 0 || closer(t, i, h))) {
                    h->tri = i; h->t = t; h->u = u; h->v = v;
                }
            }
        } else {
            stack[sp++] = n->right;
            stack[sp++] = n->left;
        }
    }
}

static void intersect(const oscene* S, v3 o, v3 d, double tmax, ohit* h) {
    if (S->use_bvh) intersect_bvh(S, o, d, tmax, h);
    else intersect_brute(S, o, d, tmax, h);
}

static int occluded(const oscene* S, v3 o, v3 d, double tmax) {
    ohit h;
    intersect(S, o, d, tmax, &h);
    return h.tri >= 0;
}

/* closest hit for n rays (o, d, tmax, pad per ray); mode 0 = scene's own structure,
 * 1 = brute force */
void oracle_intersect(void* hs, const double* rays, int n, int brute, int* tri_out,
                      double* t_out, double* uv_out) {
    const oscene* S = (const oscene*)hs;
    for (int i = 0; i < n; ++i) {
        const double* r = &rays[8 * i];
        ohit h;
        v3 o = mk(r[0], r[1], r[2]), d = mk(r[3], r[4], r[5]);
        if (brute) intersect_brute(S, o, d, r[6], &h);
        else intersect(S, o, d, r[6], &h);
        tri_out[i] = h.tri;
        t_out[i] = h.tri >= 0 ? h.t : INFINITY;
        uv_out[2 * i] = h.u;
        uv_out[2 * i + 1] = h.v;
    }
}

/* ------------------------------------------------------------------------------------ */
/* Environment map: lat-long, +y up; u = 0.5 + atan2(dx, -dz)/(2 pi), v = acos(dy)/pi     */
/* ------------------------------------------------------------------------------------ */
static void env_texel(const oscene* S, v3 d, int* x, int* y) {
    double u = 0.5 + atan2(d.x, -d.z) / (2.0 * M_PI);
    double dy = d.y < -1.0 ? -1.0 : (d.y > 1.0 ? 1.0 : d.y);
    double v = acos(dy) / M_PI;
    int ix = (int)floor(u * S->env_w), iy = (int)floor(v * S->env_h);
    if (ix < 0) ix = 0;
    if (ix > S->env_w - 1) ix = S->env_w - 1;
    if (iy < 0) iy = 0;
    if (iy > S->env_h - 1) iy = S->env_h - 1;
    *x = ix; *y = iy;
}

static v3 env_radiance(const oscene* S, v3 d) {
    int x, y;
    env_texel(S, d, &x, &y);
    const double* t = &S->env[3 * ((size_t)y * S->env_w + x)];
    return mk(t[0], t[1], t[2]);
}

/* solid-angle density of sampling direction d from the environment distribution */
static double env_pdf(const oscene* S, v3 d) {
    if (S->env_total <= 0.0) return 0.0;
    int x, y;
    env_texel(S, d, &x, &y);
    double s = sqrt(fmax(0.0, 1.0 - d.y * d.y));
    if (s <= 0.0) return 0.0;
    double pdf_uv = S->env_w_tex[(size_t)y * S->env_w + x] / S->env_total *
                    (double)S->env_w * S->env_h;
    return pdf_uv / (2.0 * M_PI * M_PI * s);
}

/* largest i in [0, n-1] with cdf[i] <= u (cdf has n+1 entries, cdf[0] = 0) */
static int cdf_find(const double* cdf, int n, double u) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (cdf[mid] <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

static int env_sample(const oscene* S, double u3, double u4, v3* d, double* pdf, v3* L) {
    if (S->env_total <= 0.0) return 0;
    int w = S->env_w, h = S->env_h;
    int y = cdf_find(S->env_marg, h, u3);
    double m0 = S->env_marg[y], m1 = S->env_marg[y + 1];
    double dv = m1 > m0 ? (u3 - m0) / (m1 - m0) : 0.5;
    const double* cd = &S->env_cond[(size_t)y * (w + 1)];
    int x = cdf_find(cd, w, u4);
    double c0 = cd[x], c1 = cd[x + 1];
    double du = c1 > c0 ? (u4 - c0) / (c1 - c0) : 0.5;
    double u = (x + du) / w, v = (y + dv) / h;
    double theta = v * M_PI, phi = (u - 0.5) * 2.0 * M_PI;
    double st = sin(theta);
    if (st <= 0.0) return 0;
    *d = mk(st * sin(phi), cos(theta), -st * cos(phi));
    double pdf_uv = S->env_w_tex[(size_t)y * w + x] / S->env_total * (double)w * h;
    *pdf = pdf_uv / (2.0 * M_PI * M_PI * st);
    const double* t = &S->env[3 * ((size_t)y * w + x)];
    *L = mk(t[0], t[1], t[2]);
    return *pdf > 0.0;
}

int oracle_env_sample(void* hs, double u3, double u4, double d_out[3], double* pdf,
                      double L_out[3]) {
    v3 d, L;
    int ok = env_sample((oscene*)hs, u3, u4, &d, pdf, &L);
    if (ok) {
        d_out[0] = d.x; d_out[1] = d.y; d_out[2] = d.z;
        L_out[0] = L.x; L_out[1] = L.y; L_out[2] = L.z;
    }
    return ok;
}
double oracle_env_pdf(void* hs, const double d[3]) {
    return env_pdf((oscene*)hs, mk(d[0], d[1], d[2]));
}

/* ------------------------------------------------------------------------------------ */
/* Path tracer                                                                             */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    v3 origin, target, up;
    double vfov_deg;
    int width, height;
    double lens_radius, focus_distance;   /* thin lens; radius 0 = pinhole */
} ocam;

typedef struct {
    long long ext_rays, shadow_rays, nan_dropped, rr_terminated, paths;
} ostats;

/* orthonormal basis around n (Duff et al., JCGT 6(1), 2017) */
static void onb(v3 n, v3* t, v3* b) {
    double s = n.z >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (s + n.z);
    double c = n.x * n.y * a;
    *t = mk(1.0 + s * n.x * n.x * a, s * c, -s * n.x);
    *b = mk(c, s + n.y * n.y * a, -n.y);
}

/* Tangent frame of an anisotropic surface (reading: the interface carries no vertex
 * tangents, so the tangent is the triangle's first edge e1 = p1 - p0 projected into the
 * shading plane, then turned about n by `rot` turns): t0 = normalize(e1 - n (n.e1)),
 * t = cos(2 pi rot) t0 + sin(2 pi rot) (n x t0), b = n x t.  (t, b, n) is right-handed. */
static void tangent_frame(v3 n, v3 e1, double rot, v3* t, v3* b) {
    v3 t0 = sub(e1, scl(n, dot(n, e1)));
    double l2 = dot(t0, t0);
    if (!(l2 > 0.0)) { onb(n, t, b); return; }
    t0 = scl(t0, 1.0 / sqrt(l2));
    v3 b0 = cross(n, t0);
    double c = cos(2.0 * M_PI * rot), s = sin(2.0 * M_PI * rot);
    *t = add(scl(t0, c), scl(b0, s));
    *b = cross(n, *t);
}
void oracle_tangent_frame(const double n[3], const double e1[3], double rot, double t[3], double b[3]) {
    v3 tt, bb;
    tangent_frame(mk(n[0], n[1], n[2]), mk(e1[0], e1[1], e1[2]), rot, &tt, &bb);
    t[0] = tt.x; t[1] = tt.y; t[2] = tt.z;
    b[0] = bb.x; b[1] = bb.y; b[2] = bb.z;
}

static inline double power_heuristic(double pa, double pb) {
    double a2 = pa * pa, b2 = pb * pb;
    return a2 + b2 > 0.0 ? a2 / (a2 + b2) : 0.0;
}

static v3 offset_origin(const oscene* S, v3 x, v3 ng, v3 dir) {
    double s = dot(dir, ng) > 0.0 ? 1.0 : -1.0;
    return add(x, scl(ng, s * S->eps));
}

static inline double U(uint32_t p, uint32_t s, uint32_t k, uint32_t dim, uint64_t seed) {
    return oracle_uniform(p, s, k, dim, seed);
}

/* Concentric map of the unit square onto the unit disk (Shirley and Chiu 1997): square rings
 * go to disk rings, so the map preserves relative area and uniform points stay uniform. */
static void concentric_disk(double u0, double u1, double* x, double* y) {
    double a = 2.0 * u0 - 1.0, b = 2.0 * u1 - 1.0;
    if (a == 0.0 && b == 0.0) { *x = 0.0; *y = 0.0; return; }
    double r, phi;
    if (fabs(a) > fabs(b)) { r = a; phi = 0.25 * M_PI * (b / a); }
    else { r = b; phi = 0.5 * M_PI - 0.25 * M_PI * (a / b); }
    *x = r * cos(phi);
    *y = r * sin(phi);
}

/* The camera ray of pixel (px, py), sample s: jitter inside the pixel (box filter).  Pinhole
 * when lens_radius = 0; else a thin lens (depth of field, a future-work item of Sec. 6.3): the lens
 * point, on the disk of that radius in the (right, up) plane, comes from dimensions 12-13 by
 * the concentric map, and the ray aims at the point where the pinhole ray of the same
 * jitter meets the plane of focus, perpendicular to the view direction at focus_distance. */
static void camera_ray(const ocam* c, int px, int py, uint32_t s, uint64_t seed, v3* o, v3* d) {
    uint32_t p = (uint32_t)(py * c->width + px);
    double u0 = U(p, s, 0, DIM_CAM_X, seed), u1 = U(p, s, 0, DIM_CAM_Y, seed);
    v3 fwd = normalize(sub(c->target, c->origin));
    v3 right = normalize(cross(fwd, c->up));
    v3 up = cross(right, fwd);
    double th = tan(0.5 * c->vfov_deg * M_PI / 180.0);
    double aspect = (double)c->width / (double)c->height;
    double nx = (2.0 * (px + u0) / c->width - 1.0) * aspect * th;
    double ny = (1.0 - 2.0 * (py + u1) / c->height) * th;
    v3 dp = normalize(add(add(fwd, scl(right, nx)), scl(up, ny)));
    if (c->lens_radius > 0.0) {
        double lx, ly;
        concentric_disk(U(p, s, 0, DIM_LENS_U, seed), U(p, s, 0, DIM_LENS_V, seed), &lx, &ly);
        v3 focus = add(c->origin, scl(dp, c->focus_distance / dot(dp, fwd)));
        v3 lens = add(c->origin, add(scl(right, c->lens_radius * lx), scl(up, c->lens_radius * ly)));
        *o = lens;
        *d = normalize(sub(focus, lens));
        return;
    }
    *o = c->origin;
    *d = dp;
}

/* Radiance of one path (pixel p, sample s).  Recursion written as a loop over vertices k.
 * Readings: pbrt-style depth (max_depth = number of BSDF-sampled bounces); next-event
 * estimation at every vertex with a non-delta lobe, env chosen with probability 1/2 when
 * both kinds of light exist, quads uniformly; power heuristic (beta = 2); roulette from
 * vertex 3 with q = min(0.95, max beta); lights are black emitters, emission front side. */
/* flags: bit 0 = no next-event estimation (BSDF sampling only, emission weight 1),
 *        bit 1 = no Russian roulette */
enum { FLAG_NO_NEE = 1, FLAG_NO_RR = 2 };

/* ---- ReSTIR DI at the primary vertex ------------------------------------------------ */
/* The paper points to reservoir resampling for many-light direct illumination as future    */
/* work (Sec. 2, Sec. 6.3) without fixing an algorithm; this follows Bitterli et al. 2020:  */
/*  1. initial candidates: M light samples y_i from the NEE light sampler (source pdf p_i, */
/*     area measure on quads, solid angle for the environment), resampled with the cheap   */
/*     target p0(y) = lum(L_e(y)) G(y) |cos| (G = cos_l / d^2 on a quad, 1 for the          */
/*     environment) on the side of the surface it scatters to (above it, or both sides if  */
/*     it transmits): its support holds that of the contribution, so the reservoir stays    */
/*     unbiased (generalised RIS); a one-sample weighted reservoir keeps y_i with           */
/*     probability w_i / sum_j w_j, w_i = p0(y_i) / p_i, and W = sum w / (M p0(y));         */
/*  2. one spatial pass: K neighbours of the same sample index inside the window (offsets  */
/*     uniform in a square of half-width R, rejected off-window, on the pixel itself, with  */
/*     no surface, normal cosine < 0.9 or depth differing by > 10 %); this pixel's and the  */
/*     neighbours' initial reservoirs are resampled with the full target p^_q (luminance of */
/*     the unshadowed contribution f(wo, w_y) L_e(y) |cos| G(y)) at this pixel q,           */
/*     w_j = p^_q(y_j) W_j M_j, and the result is weighted unbiasedly: W = sum w /          */
/*     (Z p^_q(y)), Z = sum of M_j over the combined reservoirs whose own initial target p0 */
/*     is positive at y (the "1/Z" weights count the reservoirs that could have drawn y);   */
/*  3. vertex 0 of the path shades that sample: f L_e |cos| G V W with one shadow ray, in   */
/*     place of next-event estimation; a BSDF-sampled hit of a quad or the environment at   */
/*     vertex 1 then counts with weight 0 (unless vertex 0 sampled a delta lobe), since the */
/*     reservoir already estimates all light reaching vertex 0.                             */
/*  4. optionally, at every later vertex k >= 1, next-event estimation by resampled        */
/*     importance sampling of L candidates with the same cheap target (no spatial reuse;   */
/*     stream RESTIR_LATER + k), and a BSDF-sampled light hit after such a vertex counts    */
/*     with weight 0 as well.                                                               */
/* Random numbers: candidate i uses (pixel, sample, RESTIR_CANDIDATES, dims 4i..4i+3) for   */
/* light pick, u, v, selection; neighbour j uses (pixel, sample, RESTIR_SPATIAL, 4j..4j+2)  */
/* for dx, dy (the raw 32-bit words, w * (2R+1) >> 32 - R: integer arithmetic, so both      */
/* sides pick the same pixel) and selection.                                                */
#define RESTIR_CANDIDATES 0xFFFF0001u
#define RESTIR_SPATIAL 0xFFFF0002u
#define RESTIR_LATER 0xFFFF0100u   /* + vertex index: resampled light candidates at vertex k >= 1 */
enum { LIGHT_NONE = -2, LIGHT_ENV = -1 };

typedef struct {
    int valid;               /* a scattering surface that next-event estimation would shade */
    v3 x, ng, n, tt, bb, wo_w, wo;
    double t;
    int front;
    int transmits;           /* scatters to both sides: (1 - metalness) transmission_weight > 0 */
    closure C;
} osurf;

typedef struct {
    int light;               /* quad index, LIGHT_ENV or LIGHT_NONE */
    v3 y;                    /* point on the quad, or direction towards the environment */
    double W, M, phat;
} oresv;

static uint32_t philox_word(uint32_t p, uint32_t s, uint32_t k, uint32_t dim, uint64_t seed) {
    uint32_t ctr[4] = {p, s, k, dim >> 2};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    return out[dim & 3u];
}

/* unshadowed contribution of light sample (light, y) at surface g; returns p^ = its luminance */
static double restir_target(const oscene* S, const osurf* g, int light, v3 y, v3* c_out, v3* ld_out) {
    v3 ld, Le;
    double geo;
    *c_out = splat(0.0);
    if (light >= 0) {
        v3 to = sub(y, g->x);
        double d2 = dot(to, to);
        if (!(d2 > 0.0)) return 0.0;
        ld = scl(to, 1.0 / sqrt(d2));
        double cl = -dot(ld, S->q_n[light]);
        if (!(cl > 0.0 || (S->q_two_sided[light] && cl < 0.0))) return 0.0;
        Le = S->q_L[light];
        geo = fabs(cl) / d2;
    } else if (light == LIGHT_ENV) {
        ld = y;
        Le = env_radiance(S, ld);
        geo = 1.0;
    } else {
        return 0.0;
    }
    v3 wl = mk(dot(ld, g->tt), dot(ld, g->bb), dot(ld, g->n));
    v3 f;
    double pdf;
    closure_eval(&g->C, g->wo, wl, &f, &pdf);
    v3 c = scl(hmul(f, Le), fabs(wl.z) * geo);
    *c_out = c;
    *ld_out = ld;
    double ph = lum(c);
    return ph > 0.0 && isfinite(ph) ? ph : 0.0;
}

/* cheap target p0 of the initial candidates: lum(L_e) G |cos| where the surface scatters */
static double restir_target0(const oscene* S, const osurf* g, int light, v3 y) {
    v3 ld, Le;
    double geo;
    if (light >= 0) {
        v3 to = sub(y, g->x);
        double d2 = dot(to, to);
        if (!(d2 > 0.0)) return 0.0;
        ld = scl(to, 1.0 / sqrt(d2));
        double cl = -dot(ld, S->q_n[light]);
        if (!(cl > 0.0 || (S->q_two_sided[light] && cl < 0.0))) return 0.0;
        Le = S->q_L[light];
        geo = fabs(cl) / d2;
    } else if (light == LIGHT_ENV) {
        ld = y;
        Le = env_radiance(S, ld);
        geo = 1.0;
    } else {
        return 0.0;
    }
    double c = dot(ld, g->n);
    if (!(c > 0.0) && !(g->transmits && c < 0.0)) return 0.0;
    double ph = lum(Le) * geo * fabs(c);
    return ph > 0.0 && isfinite(ph) ? ph : 0.0;
}

static void restir_initial(const oscene* S, const osurf* g, uint32_t p, uint32_t s, uint32_t stream, uint64_t seed,
                           int M, double p_env, oresv* R) {
    R->light = LIGHT_NONE;
    R->y = splat(0.0);
    R->W = 0.0;
    R->M = (double)M;
    R->phat = 0.0;
    double wsum = 0.0;
    for (int i = 0; i < M; ++i) {
        double u_pick = U(p, s, stream, 4u * i, seed);
        double u = U(p, s, stream, 4u * i + 1, seed);
        double v = U(p, s, stream, 4u * i + 2, seed);
        double u_sel = U(p, s, stream, 4u * i + 3, seed);
        int light;
        v3 y;
        double src;
        if (u_pick < p_env) {
            v3 Ld;
            double pe;
            if (!env_sample(S, u, v, &y, &pe, &Ld)) continue;
            light = LIGHT_ENV;
            src = p_env * pe;
        } else {
            int l = (int)floor((u_pick - p_env) / (1.0 - p_env) * S->n_quads);
            if (l > S->n_quads - 1) l = S->n_quads - 1;
            light = l;
            y = add(add(S->q_p0[l], scl(S->q_e1[l], u)), scl(S->q_e2[l], v));
            src = (1.0 - p_env) / S->n_quads / S->q_area[l];
        }
        if (!(src > 0.0)) continue;
        double ph = restir_target0(S, g, light, y);
        double w = ph / src;
        if (!(w > 0.0)) continue;
        wsum += w;
        if (u_sel * wsum < w) {
            R->light = light;
            R->y = y;
            R->phat = ph;
        }
    }
    if (R->light != LIGHT_NONE && R->phat > 0.0) R->W = wsum / (R->M * R->phat);
}

typedef struct {
    const oscene* S;
    const ocam* cam;
    int x0, y0, cw, ch, M, K, R, Lm;
    int max_depth, flags;
    uint32_t s;
    uint64_t seed;
    osurf* surf;
    oresv* init;
    oresv* fin;
    int tid, nthreads;
} restir_job;

/* pass 1: the primary surface of every pixel of the window and its initial reservoir */
static void* restir_pass_initial(void* arg) {
    restir_job* J = (restir_job*)arg;
    const oscene* S = J->S;
    int has_env = S->env_w > 0 && S->env_total > 0.0;
    double p_env = has_env ? (S->n_quads > 0 ? 0.5 : 1.0) : 0.0;
    for (int ry = J->tid; ry < J->ch; ry += J->nthreads)
        for (int rx = 0; rx < J->cw; ++rx) {
            size_t i = (size_t)ry * J->cw + rx;
            osurf* g = &J->surf[i];
            memset(g, 0, sizeof(*g));
            J->init[i].light = LIGHT_NONE;
            J->init[i].W = J->init[i].M = J->init[i].phat = 0.0;
            int px = J->x0 + rx, py = J->y0 + ry;
            uint32_t p = (uint32_t)(py * J->cam->width + px);
            v3 o, d;
            camera_ray(J->cam, px, py, J->s, J->seed, &o, &d);
            ohit h;
            intersect(S, o, d, INFINITY, &h);
            if (h.tri < 0 || J->max_depth == 0) continue;
            int mid = S->tri_mat[h.tri];
            if (mid < 0) continue;
            const omat* m = &S->mats[mid];
            v3 p0 = S->tv[3 * h.tri], p1 = S->tv[3 * h.tri + 1], p2 = S->tv[3 * h.tri + 2];
            g->x = add(o, scl(d, h.t));
            g->ng = normalize(cross(sub(p1, p0), sub(p2, p0)));
            g->wo_w = scl(d, -1.0);
            g->front = dot(g->wo_w, g->ng) > 0.0;
            g->n = g->front ? g->ng : scl(g->ng, -1.0);
            if (m->spec_aniso > 0.0) tangent_frame(g->n, sub(p1, p0), m->spec_rot, &g->tt, &g->bb);
            else onb(g->n, &g->tt, &g->bb);
            g->wo = mk(dot(g->wo_w, g->tt), dot(g->wo_w, g->bb), dot(g->wo_w, g->n));
            g->t = h.t;
            g->transmits = (1.0 - m->metalness) * m->trans_weight > 0.0;
            closure_setup(&g->C, m, g->front, g->wo.z);
            g->valid = g->C.has_smooth && (has_env || S->n_quads > 0);
            if (g->valid) restir_initial(S, g, p, J->s, RESTIR_CANDIDATES, J->seed, J->M, p_env, &J->init[i]);
        }
    return NULL;
}

/* pass 2: spatial reuse over K neighbours with the 1/Z weights */
static void* restir_pass_spatial(void* arg) {
    restir_job* J = (restir_job*)arg;
    const oscene* S = J->S;
    const int side = 2 * J->R + 1;
    for (int ry = J->tid; ry < J->ch; ry += J->nthreads)
        for (int rx = 0; rx < J->cw; ++rx) {
            size_t i = (size_t)ry * J->cw + rx;
            const osurf* g = &J->surf[i];
            oresv* F = &J->fin[i];
            *F = J->init[i];
            if (!g->valid) continue;
            int px = J->x0 + rx, py = J->y0 + ry;
            uint32_t p = (uint32_t)(py * J->cam->width + px);
            const oresv* R0 = &J->init[i];
            v3 c0, ld0;
            double wsum = restir_target(S, g, R0->light, R0->y, &c0, &ld0) * R0->W * R0->M;
            double Msum = R0->M;
            int light = R0->light;
            v3 y = R0->y;
            size_t used[64];
            int n_used = 0;
            for (int j = 0; j < J->K && j < 64; ++j) {
                uint32_t wx = philox_word(p, J->s, RESTIR_SPATIAL, 4u * j, J->seed);
                uint32_t wy = philox_word(p, J->s, RESTIR_SPATIAL, 4u * j + 1, J->seed);
                double u_sel = U(p, J->s, RESTIR_SPATIAL, 4u * j + 2, J->seed);
                int dx = (int)(((uint64_t)wx * (uint32_t)side) >> 32) - J->R;
                int dy = (int)(((uint64_t)wy * (uint32_t)side) >> 32) - J->R;
                int nx = rx + dx, ny = ry + dy;
                if ((dx == 0 && dy == 0) || nx < 0 || ny < 0 || nx >= J->cw || ny >= J->ch) continue;
                size_t k = (size_t)ny * J->cw + nx;
                const osurf* gn = &J->surf[k];
                if (!gn->valid) continue;
                if (dot(gn->n, g->n) < 0.9 || fabs(gn->t - g->t) > 0.1 * g->t) continue;
                const oresv* Rn = &J->init[k];
                used[n_used++] = k;
                Msum += Rn->M;
                v3 c, ld;
                double ph = restir_target(S, g, Rn->light, Rn->y, &c, &ld);
                double w = ph * Rn->W * Rn->M;
                if (!(w > 0.0)) continue;
                wsum += w;
                if (u_sel * wsum < w) {
                    light = Rn->light;
                    y = Rn->y;
                }
            }
            (void)Msum;
            v3 c, ld;
            double ph = restir_target(S, g, light, y, &c, &ld);
            double Z = restir_target0(S, g, light, y) > 0.0 ? R0->M : 0.0;
            for (int u = 0; u < n_used; ++u)
                if (restir_target0(S, &J->surf[used[u]], light, y) > 0.0) Z += J->init[used[u]].M;
            F->light = light;
            F->y = y;
            F->phat = ph;
            F->M = Z;
            F->W = (ph > 0.0 && Z > 0.0) ? wsum / (Z * ph) : 0.0;
        }
    return NULL;
}

static v3 trace_path_r(const oscene* S, const ocam* cam, int px, int py, uint32_t s,
                       int max_depth, uint64_t seed, int flags, ostats* st, int restir, int later_m,
                       const oresv* R0, const osurf* g0);

static v3 trace_path(const oscene* S, const ocam* cam, int px, int py, uint32_t s,
                     int max_depth, uint64_t seed, int flags, ostats* st) {
    return trace_path_r(S, cam, px, py, s, max_depth, seed, flags, st, 0, 0, NULL, NULL);
}

/* one path; with `restir`, vertex 0 shades the reservoir R0 (its surface g0) instead of NEE,
 * and with later_m > 0 the later vertices resample later_m light candidates */
static v3 trace_path_r(const oscene* S, const ocam* cam, int px, int py, uint32_t s,
                       int max_depth, uint64_t seed, int flags, ostats* st, int restir, int later_m,
                       const oresv* R0, const osurf* g0) {
    uint32_t p = (uint32_t)(py * cam->width + px);
    v3 o, d;
    camera_ray(cam, px, py, s, seed, &o, &d);
    v3 L = splat(0.0), beta = splat(1.0);
    int nee = !(flags & FLAG_NO_NEE);
    int prev_delta = 1;
    double prev_pdf = 0.0;
    int has_env = S->env_w > 0 && S->env_total > 0.0;
    double p_env = has_env ? (S->n_quads > 0 ? 0.5 : 1.0) : 0.0;
    for (int k = 0;; ++k) {
        ohit h;
        intersect(S, o, d, INFINITY, &h);
        st->ext_rays++;
        if (h.tri < 0) {
            if (has_env) {
                v3 Le = env_radiance(S, d);
                double w = 1.0;
                if (!prev_delta && nee)
                    w = (restir && (k == 1 || later_m > 0)) ? 0.0 : power_heuristic(prev_pdf, p_env * env_pdf(S, d));
                L = add(L, scl(hmul(beta, Le), w));
            }
            break;
        }
        v3 x = add(o, scl(d, h.t));
        v3 p0 = S->tv[3 * h.tri], p1 = S->tv[3 * h.tri + 1], p2 = S->tv[3 * h.tri + 2];
        v3 ng = normalize(cross(sub(p1, p0), sub(p2, p0)));
        v3 wo_w = scl(d, -1.0);
        int front = dot(wo_w, ng) > 0.0;
        int mid = S->tri_mat[h.tri];
        if (mid < 0) {
            int l = -1 - mid;
            double cl = dot(wo_w, S->q_n[l]);
            if (cl > 0.0 || (S->q_two_sided[l] && cl < 0.0)) {
                double w = 1.0;
                if (!prev_delta && nee) {
                    double pl = (1.0 - p_env) / S->n_quads * h.t * h.t / (S->q_area[l] * fabs(cl));
                    w = (restir && (k == 1 || later_m > 0)) ? 0.0 : power_heuristic(prev_pdf, pl);
                }
                L = add(L, scl(hmul(beta, S->q_L[l]), w));
            }
            break;
        }
        const omat* m = &S->mats[mid];
        if (m->emission > 0.0 && front) L = add(L, scl(hmul(beta, m->emission_color), m->emission));
        if (k == max_depth) break;

        v3 n = front ? ng : scl(ng, -1.0);
        v3 tt, bb;
        if (m->spec_aniso > 0.0) tangent_frame(n, sub(p1, p0), m->spec_rot, &tt, &bb);
        else onb(n, &tt, &bb);
        v3 wo = mk(dot(wo_w, tt), dot(wo_w, bb), dot(wo_w, n));
        closure C;
        closure_setup(&C, m, front, wo.z);

        if (restir && k == 0) {
            /* the reservoir's sample in place of next-event estimation */
            if (g0 && g0->valid && R0 && R0->light != LIGHT_NONE && R0->W > 0.0) {
                v3 c, ld;
                double ph = restir_target(S, g0, R0->light, R0->y, &c, &ld);
                if (ph > 0.0) {
                    v3 so = offset_origin(S, x, ng, ld);
                    v3 sd = ld;
                    double tmax = INFINITY;
                    if (R0->light >= 0) {
                        v3 to = sub(R0->y, so);
                        double dl = length(to);
                        sd = scl(to, 1.0 / dl);
                        tmax = (1.0 - 1e-4) * dl;
                    }
                    st->shadow_rays++;
                    if (!occluded(S, so, sd, tmax)) L = add(L, scl(hmul(beta, c), R0->W));
                }
            }
        } else if (restir && later_m > 0 && C.has_smooth && (has_env || S->n_quads > 0)) {
            /* resampled light candidates at a later vertex */
            osurf gk;
            gk.valid = 1;
            gk.x = x; gk.ng = ng; gk.n = n; gk.tt = tt; gk.bb = bb; gk.wo_w = wo_w; gk.wo = wo;
            gk.t = h.t; gk.front = front;
            gk.transmits = (1.0 - m->metalness) * m->trans_weight > 0.0;
            gk.C = C;
            oresv Rk;
            restir_initial(S, &gk, p, s, RESTIR_LATER + (uint32_t)k, seed, later_m, p_env, &Rk);
            if (Rk.light != LIGHT_NONE && Rk.W > 0.0) {
                v3 c, ld;
                if (restir_target(S, &gk, Rk.light, Rk.y, &c, &ld) > 0.0) {
                    v3 so = offset_origin(S, x, ng, ld);
                    v3 sd = ld;
                    double tmax = INFINITY;
                    if (Rk.light >= 0) {
                        v3 to = sub(Rk.y, so);
                        double dl = length(to);
                        sd = scl(to, 1.0 / dl);
                        tmax = (1.0 - 1e-4) * dl;
                    }
                    st->shadow_rays++;
                    if (!occluded(S, so, sd, tmax)) L = add(L, scl(hmul(beta, c), Rk.W));
                }
            }
        } else if (nee && C.has_smooth && (has_env || S->n_quads > 0)) {
            /* next-event estimation */
            double u2 = U(p, s, (uint32_t)k, DIM_LIGHT_PICK, seed);
            double u3 = U(p, s, (uint32_t)k, DIM_LIGHT_U, seed);
            double u4 = U(p, s, (uint32_t)k, DIM_LIGHT_V, seed);
            v3 ld, Le = splat(0.0), ly = splat(0.0);
            double pl = 0.0;
            int ok = 0, to_quad = 0;
            if (u2 < p_env) {
                double pe;
                if (env_sample(S, u3, u4, &ld, &pe, &Le)) {
                    pl = p_env * pe;
                    ok = 1;
                }
            } else {
                int l = (int)floor((u2 - p_env) / (1.0 - p_env) * S->n_quads);
                if (l > S->n_quads - 1) l = S->n_quads - 1;
                v3 y = add(add(S->q_p0[l], scl(S->q_e1[l], u3)), scl(S->q_e2[l], u4));
                v3 to = sub(y, x);
                double dist2 = dot(to, to), dist = sqrt(dist2);
                ld = scl(to, 1.0 / dist);
                double cl = -dot(ld, S->q_n[l]);
                if (cl > 0.0 || (S->q_two_sided[l] && cl < 0.0)) {
                    pl = (1.0 - p_env) / S->n_quads * dist2 / (S->q_area[l] * fabs(cl));
                    Le = S->q_L[l];
                    ly = y;
                    to_quad = 1;
                    ok = 1;
                }
            }
            if (ok && pl > 0.0) {
                v3 wl = mk(dot(ld, tt), dot(ld, bb), dot(ld, n));
                v3 f;
                double pb;
                closure_eval(&C, wo, wl, &f, &pb);
                if (maxc(f) > 0.0) {
                    /* shadow ray from the offset origin; towards a quad it aims at the light
                     * point itself and stops 1e-4 (relative) short of it */
                    v3 so = offset_origin(S, x, ng, ld);
                    v3 sd = ld;
                    double tmax = INFINITY;
                    if (to_quad) {
                        v3 to = sub(ly, so);
                        double dl = length(to);
                        sd = scl(to, 1.0 / dl);
                        tmax = (1.0 - 1e-4) * dl;
                    }
                    st->shadow_rays++;
                    if (!occluded(S, so, sd, tmax)) {
                        double w = power_heuristic(pl, pb);
                        L = add(L, scl(hmul(hmul(beta, f), Le), fabs(wl.z) * w / pl));
                    }
                }
            }
        }

        /* BSDF sampling */
        double u5 = U(p, s, (uint32_t)k, DIM_LOBE, seed);
        double u6 = U(p, s, (uint32_t)k, DIM_DIR_U, seed);
        double u7 = U(p, s, (uint32_t)k, DIM_DIR_V, seed);
        double u8 = U(p, s, (uint32_t)k, DIM_REFRACT, seed);
        bsdf_sample_t bs;
        if (!closure_sample(&C, wo, u5, u6, u7, u8, &bs)) break;
        beta = hmul(beta, bs.weight);
        if (k >= 3 && !(flags & FLAG_NO_RR)) {
            double q = fmin(0.95, maxc(beta));
            if (U(p, s, (uint32_t)k, DIM_RR, seed) >= q) { st->rr_terminated++; break; }
            beta = scl(beta, 1.0 / q);
        }
        v3 wi_w = add(add(scl(tt, bs.wi.x), scl(bb, bs.wi.y)), scl(n, bs.wi.z));
        o = offset_origin(S, x, ng, wi_w);
        d = normalize(wi_w);
        prev_delta = bs.is_delta;
        prev_pdf = bs.pdf;
    }
    return L;
}

/* ---- multi-threaded rendering of a crop of the frame ---- */
typedef struct {
    const oscene* S;
    const ocam* cam;
    int x0, y0, cw, ch, row_step;
    uint32_t s0, spp;
    int max_depth;
    uint64_t seed;
    int flags;
    double* sum;          /* ch * cw * 3 */
    double* samples;      /* optional ch * cw * spp * 3 */
    int tid, nthreads;
    ostats st;
} job_t;

static void* worker(void* arg) {
    job_t* J = (job_t*)arg;
    memset(&J->st, 0, sizeof(J->st));
    for (int j = J->tid; j * J->row_step < J->ch; j += J->nthreads) {
        int ry = j * J->row_step;
        for (int rx = 0; rx < J->cw; ++rx) {
            double acc[3] = {0, 0, 0};
            for (uint32_t i = 0; i < J->spp; ++i) {
                v3 L = trace_path(J->S, J->cam, J->x0 + rx, J->y0 + ry, J->s0 + i, J->max_depth,
                                  J->seed, J->flags, &J->st);
                J->st.paths++;
                if (!isfinite(L.x) || !isfinite(L.y) || !isfinite(L.z)) {
                    J->st.nan_dropped++;
                    L = splat(0.0);
                }
                acc[0] += L.x; acc[1] += L.y; acc[2] += L.z;
                if (J->samples) {
                    double* sp = &J->samples[(((size_t)ry * J->cw + rx) * J->spp + i) * 3];
                    sp[0] = L.x; sp[1] = L.y; sp[2] = L.z;
                }
            }
            double* o = &J->sum[((size_t)ry * J->cw + rx) * 3];
            o[0] = acc[0]; o[1] = acc[1]; o[2] = acc[2];
        }
    }
    return NULL;
}

/* Render samples s0 .. s0+spp-1 of the crop [x0, x0+cw) x [y0, y0+ch) of the full frame.
 * sum_out receives the per-pixel sum of sample radiance (divide by spp for the estimate).
 * restir = NULL for next-event estimation, else {M candidates, K neighbours, radius R, L later
 * candidates}: ReSTIR DI at the primary vertex over the window (row_step is then ignored),
 * resampled next-event estimation with L candidates at later vertices if L > 0.
 * cam = origin[3], target[3], up[3], lens_radius, focus_distance; row_step > 1 renders only every row_step-th
 * row of the crop (others stay 0); flags as for trace_path.  stats_out (5 int64): extension rays, shadow rays, NaN
 * samples dropped, roulette terminations, paths. */
/* pass 3 of ReSTIR: the paths of sample J->s, vertex 0 shading the final reservoirs */
typedef struct {
    restir_job* R;
    uint32_t i, spp;
    double* sum;
    double* samples;
    ostats st;
} restir_path_job;

static void* restir_pass_paths(void* arg) {
    restir_path_job* P = (restir_path_job*)arg;
    restir_job* J = P->R;
    for (int ry = J->tid; ry < J->ch; ry += J->nthreads)
        for (int rx = 0; rx < J->cw; ++rx) {
            size_t i = (size_t)ry * J->cw + rx;
            v3 L = trace_path_r(J->S, J->cam, J->x0 + rx, J->y0 + ry, J->s, J->max_depth, J->seed, J->flags,
                                &P->st, 1, J->Lm, &J->fin[i], &J->surf[i]);
            P->st.paths++;
            if (!isfinite(L.x) || !isfinite(L.y) || !isfinite(L.z)) {
                P->st.nan_dropped++;
                L = splat(0.0);
            }
            double* o = &P->sum[i * 3];
            o[0] += L.x; o[1] += L.y; o[2] += L.z;
            if (P->samples) {
                double* sp = &P->samples[(i * P->spp + P->i) * 3];
                sp[0] = L.x; sp[1] = L.y; sp[2] = L.z;
            }
        }
    return NULL;
}

static void run_threads(void* (*fn)(void*), void* jobs, size_t job_size, int nthreads) {
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    for (int t = 0; t < nthreads; ++t) {
        void* j = (char*)jobs + job_size * (size_t)t;
        if (nthreads == 1) fn(j);
        else pthread_create(&th[t], NULL, fn, j);
    }
    if (nthreads > 1)
        for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
}

static void render_restir(const oscene* S, const ocam* cam, int x0, int y0, int cw, int ch, uint32_t s0,
                          uint32_t spp, int max_depth, uint64_t seed, int flags, int nthreads, const int* rp,
                          double* sum_out, double* samples_out, long long* tot) {
    size_t npx = (size_t)cw * ch;
    osurf* surf = (osurf*)calloc(npx, sizeof(osurf));
    oresv* init = (oresv*)calloc(npx, sizeof(oresv));
    oresv* fin = (oresv*)calloc(npx, sizeof(oresv));
    restir_job* jobs = (restir_job*)calloc((size_t)nthreads, sizeof(restir_job));
    restir_path_job* pj = (restir_path_job*)calloc((size_t)nthreads, sizeof(restir_path_job));
    for (uint32_t i = 0; i < spp; ++i) {
        for (int t = 0; t < nthreads; ++t) {
            restir_job* J = &jobs[t];
            J->S = S; J->cam = cam; J->x0 = x0; J->y0 = y0; J->cw = cw; J->ch = ch;
            J->M = rp[0]; J->K = rp[1]; J->R = rp[2]; J->Lm = rp[3];
            J->max_depth = max_depth; J->flags = flags; J->s = s0 + i; J->seed = seed;
            J->surf = surf; J->init = init; J->fin = fin; J->tid = t; J->nthreads = nthreads;
            pj[t].R = J; pj[t].i = i; pj[t].spp = spp; pj[t].sum = sum_out; pj[t].samples = samples_out;
        }
        run_threads(restir_pass_initial, jobs, sizeof(restir_job), nthreads);
        run_threads(restir_pass_spatial, jobs, sizeof(restir_job), nthreads);
        run_threads(restir_pass_paths, pj, sizeof(restir_path_job), nthreads);
    }
    for (int t = 0; t < nthreads; ++t) {
        tot[0] += pj[t].st.ext_rays; tot[1] += pj[t].st.shadow_rays;
        tot[2] += pj[t].st.nan_dropped; tot[3] += pj[t].st.rr_terminated;
        tot[4] += pj[t].st.paths;
    }
    free(surf); free(init); free(fin); free(jobs); free(pj);
}

void oracle_render(void* hs, const double* cam9, double vfov_deg, int width, int height,
                   int x0, int y0, int cw, int ch, uint32_t s0, uint32_t spp, int max_depth,
                   uint64_t seed, int flags, int nthreads, int row_step, double* sum_out,
                   double* samples_out, long long* stats_out, const int* restir) {
    ocam cam;
    cam.origin = mk(cam9[0], cam9[1], cam9[2]);
    cam.target = mk(cam9[3], cam9[4], cam9[5]);
    cam.up = mk(cam9[6], cam9[7], cam9[8]);
    cam.vfov_deg = vfov_deg;
    cam.width = width;
    cam.height = height;
    cam.lens_radius = cam9[9];
    cam.focus_distance = cam9[10];
    if (nthreads < 1) nthreads = 1;
    if (row_step < 1) row_step = 1;
    memset(sum_out, 0, sizeof(double) * 3 * (size_t)cw * ch);
    if (restir) {
        /* every pixel of the window takes part in the spatial pass: row_step must be 1 */
        long long tot[5] = {0, 0, 0, 0, 0};
        render_restir((const oscene*)hs, &cam, x0, y0, cw, ch, s0, spp, max_depth, seed, flags, nthreads, restir,
                      sum_out, samples_out, tot);
        if (stats_out) memcpy(stats_out, tot, sizeof(tot));
        return;
    }
    job_t* jobs = (job_t*)calloc((size_t)nthreads, sizeof(job_t));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    for (int t = 0; t < nthreads; ++t) {
        job_t* J = &jobs[t];
        J->S = (const oscene*)hs; J->cam = &cam;
        J->x0 = x0; J->y0 = y0; J->cw = cw; J->ch = ch; J->row_step = row_step;
        J->s0 = s0; J->spp = spp; J->max_depth = max_depth; J->seed = seed; J->flags = flags;
        J->sum = sum_out; J->samples = samples_out; J->tid = t; J->nthreads = nthreads;
        if (nthreads == 1) worker(J);
        else pthread_create(&th[t], NULL, worker, J);
    }
    if (nthreads > 1)
        for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    long long tot[5] = {0, 0, 0, 0, 0};
    for (int t = 0; t < nthreads; ++t) {
        tot[0] += jobs[t].st.ext_rays; tot[1] += jobs[t].st.shadow_rays;
        tot[2] += jobs[t].st.nan_dropped; tot[3] += jobs[t].st.rr_terminated;
        tot[4] += jobs[t].st.paths;
    }
    if (stats_out) memcpy(stats_out, tot, sizeof(tot));
    free(jobs);
    free(th);
}

/* camera ray of one pixel/sample, for the ray-generation parity check */
void oracle_camera_ray(const double* cam9, double vfov_deg, int width, int height, int px,
                       int py, uint32_t s, uint64_t seed, double o_out[3], double d_out[3]) {
    ocam cam;
    cam.origin = mk(cam9[0], cam9[1], cam9[2]);
    cam.target = mk(cam9[3], cam9[4], cam9[5]);
    cam.up = mk(cam9[6], cam9[7], cam9[8]);
    cam.vfov_deg = vfov_deg;
    cam.width = width;
    cam.height = height;
    cam.lens_radius = cam9[9];
    cam.focus_distance = cam9[10];
    v3 o, d;
    camera_ray(&cam, px, py, s, seed, &o, &d);
    o_out[0] = o.x; o_out[1] = o.y; o_out[2] = o.z;
    d_out[0] = d.x; d_out[1] = d.y; d_out[2] = d.z;
}

/* Primary-hit features for the regression denoiser (inputs of BMFR, Koskela et al. 2019;
 * the paper lists a denoiser as future work, Sec. 6.3).  For every pixel of the crop, the mean
 * over samples s0 .. s0+spp-1 (the render's own camera rays) of the first hit's shading normal
 * (turned towards the camera), position and albedo, and the fraction of those samples whose
 * first hit is a scattering surface (a miss or a light quad adds nothing to the means).
 * Reading: albedo = (m + (1-m)(1-t)) bw bc + (1-m) t tc.  out (ch*cw*12): n[3], fraction,
 * p[3], 0, albedo[3], 0. */
void oracle_features(void* hs, const double* cam9, double vfov_deg, int width, int height, int x0, int y0,
                     int cw, int ch, uint32_t s0, uint32_t spp, uint64_t seed, double* out) {
    const oscene* S = (const oscene*)hs;
    ocam cam;
    cam.origin = mk(cam9[0], cam9[1], cam9[2]);
    cam.target = mk(cam9[3], cam9[4], cam9[5]);
    cam.up = mk(cam9[6], cam9[7], cam9[8]);
    cam.vfov_deg = vfov_deg;
    cam.width = width;
    cam.height = height;
    cam.lens_radius = cam9[9];
    cam.focus_distance = cam9[10];
    for (int ry = 0; ry < ch; ++ry)
        for (int rx = 0; rx < cw; ++rx) {
            double acc[12] = {0};
            for (uint32_t i = 0; i < spp; ++i) {
                v3 o, d;
                camera_ray(&cam, x0 + rx, y0 + ry, s0 + i, seed, &o, &d);
                ohit h;
                intersect(S, o, d, INFINITY, &h);
                if (h.tri < 0 || S->tri_mat[h.tri] < 0) continue;
                const omat* m = &S->mats[S->tri_mat[h.tri]];
                v3 p0 = S->tv[3 * h.tri], p1 = S->tv[3 * h.tri + 1], p2 = S->tv[3 * h.tri + 2];
                v3 ng = normalize(cross(sub(p1, p0), sub(p2, p0)));
                v3 n = dot(scl(d, -1.0), ng) > 0.0 ? ng : scl(ng, -1.0);
                v3 x = add(o, scl(d, h.t));
                double mt = m->metalness, t = m->trans_weight;
                v3 a = add(scl(m->base_color, (mt + (1.0 - mt) * (1.0 - t)) * m->base_weight),
                           scl(m->trans_color, (1.0 - mt) * t));
                acc[0] += n.x; acc[1] += n.y; acc[2] += n.z; acc[3] += 1.0;
                acc[4] += x.x; acc[5] += x.y; acc[6] += x.z;
                acc[8] += a.x; acc[9] += a.y; acc[10] += a.z;
            }
            double* o12 = &out[((size_t)ry * cw + rx) * 12];
            for (int k = 0; k < 12; ++k) o12[k] = spp ? acc[k] / spp : 0.0;
        }
}

/* ---- batched forms of the BSDF entry points (n tuples, row-major arrays) ---- */
/* the batch entry points split their rows over the host's cores (rows are independent) */
typedef struct {
    const double *matp, *wo, *wi, *u;
    int front, n, tid, nthreads;
    double *f_out, *pdf_out, *wi_out, *weight_out;
    int *delta_out, *ok_out;
} bsdf_batch_job;

static void* bsdf_eval_rows(void* arg) {
    bsdf_batch_job* J = (bsdf_batch_job*)arg;
    for (int i = J->tid; i < J->n; i += J->nthreads)
        oracle_bsdf_eval(J->matp, J->front, &J->wo[3 * i], &J->wi[3 * i], &J->f_out[3 * i], &J->pdf_out[i]);
    return NULL;
}

static void* bsdf_sample_rows(void* arg) {
    bsdf_batch_job* J = (bsdf_batch_job*)arg;
    for (int i = J->tid; i < J->n; i += J->nthreads) {
        J->ok_out[i] = oracle_bsdf_sample(J->matp, J->front, &J->wo[3 * i], &J->u[4 * i], &J->wi_out[3 * i],
                                          &J->weight_out[3 * i], &J->pdf_out[i], &J->delta_out[i]);
        if (!J->ok_out[i]) {
            J->wi_out[3 * i] = J->wi_out[3 * i + 1] = J->wi_out[3 * i + 2] = 0.0;
            J->weight_out[3 * i] = J->weight_out[3 * i + 1] = J->weight_out[3 * i + 2] = 0.0;
        }
    }
    return NULL;
}

static void run_bsdf_batch(void* (*fn)(void*), bsdf_batch_job proto) {
    long cores = sysconf(_SC_NPROCESSORS_ONLN);
    int nt = proto.n >= 256 && cores > 1 ? (int)(cores < 64 ? cores : 64) : 1;
    bsdf_batch_job* jobs = (bsdf_batch_job*)calloc((size_t)nt, sizeof(bsdf_batch_job));
    for (int t = 0; t < nt; ++t) {
        jobs[t] = proto;
        jobs[t].tid = t;
        jobs[t].nthreads = nt;
    }
    run_threads(fn, jobs, sizeof(bsdf_batch_job), nt);
    free(jobs);
}

void oracle_bsdf_eval_batch(const double* matp, int front, int n, const double* wo,
                            const double* wi, double* f_out, double* pdf_out) {
    bsdf_batch_job J;
    memset(&J, 0, sizeof(J));
    J.matp = matp; J.front = front; J.n = n; J.wo = wo; J.wi = wi; J.f_out = f_out; J.pdf_out = pdf_out;
    run_bsdf_batch(bsdf_eval_rows, J);
}

void oracle_bsdf_sample_batch(const double* matp, int front, int n, const double* wo,
                              const double* u, double* wi_out, double* weight_out,
                              double* pdf_out, int* delta_out, int* ok_out) {
    bsdf_batch_job J;
    memset(&J, 0, sizeof(J));
    J.matp = matp; J.front = front; J.n = n; J.wo = wo; J.u = u; J.wi_out = wi_out; J.weight_out = weight_out;
    J.pdf_out = pdf_out; J.delta_out = delta_out; J.ok_out = ok_out;
    run_bsdf_batch(bsdf_sample_rows, J);
}

void oracle_uniform_batch(int n, const uint32_t* pixel, const uint32_t* sample,
                          const uint32_t* bounce, const uint32_t* dim, uint64_t seed,
                          double* out) {
    for (int i = 0; i < n; ++i) out[i] = oracle_uniform(pixel[i], sample[i], bounce[i], dim[i], seed);
}
