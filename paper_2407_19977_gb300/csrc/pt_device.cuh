// pt_device.cuh -- device building blocks of the path tracer (sm_103a).
//
// Everything here is FP32.  The formulas are the paper's method (Sec. 1.1 rendering
// equation, Sec. 5.1.2 camera and RNG, Sec. 5.1.3 BVH traversal, OpenPBR shading,
// importance sampling and Russian roulette) with the readings fixed where the paper is
// silent: Philox4x32-10 keyed by (pixel, sample, bounce, dim/4); pinhole camera with box
// filter; watertight ray/triangle test; lobe mixture with one-sample MIS; NEE to quads
// and the environment with the power heuristic; roulette from vertex 3.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define PT_PI_F 3.14159265358979323846f
#define PT_INV_PI_F 0.31830988618379067154f

// ------------------------------------------------------------------ float3 algebra
__host__ __device__ __forceinline__ float3 mk3(float x, float y, float z) { return make_float3(x, y, z); }
__host__ __device__ __forceinline__ float3 operator+(float3 a, float3 b) { return mk3(a.x + b.x, a.y + b.y, a.z + b.z); }
__host__ __device__ __forceinline__ float3 operator-(float3 a, float3 b) { return mk3(a.x - b.x, a.y - b.y, a.z - b.z); }
__host__ __device__ __forceinline__ float3 operator*(float3 a, float s) { return mk3(a.x * s, a.y * s, a.z * s); }
__host__ __device__ __forceinline__ float3 operator*(float3 a, float3 b) { return mk3(a.x * b.x, a.y * b.y, a.z * b.z); }
__host__ __device__ __forceinline__ float3 operator-(float3 a) { return mk3(-a.x, -a.y, -a.z); }
__host__ __device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__host__ __device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return mk3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ float len3(float3 a) { return sqrtf(dot3(a, a)); }
__host__ __device__ __forceinline__ float3 norm3(float3 a) { return a * (1.0f / sqrtf(dot3(a, a))); }
__host__ __device__ __forceinline__ float lum3(float3 c) { return 0.2126f * c.x + 0.7152f * c.y + 0.0722f * c.z; }
__host__ __device__ __forceinline__ float max3(float3 c) { return fmaxf(c.x, fmaxf(c.y, c.z)); }
__host__ __device__ __forceinline__ float3 splat3(float s) { return mk3(s, s, s); }
__host__ __device__ __forceinline__ float comp3(float3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }
__host__ __device__ __forceinline__ float3 xyz(float4 a) { return mk3(a.x, a.y, a.z); }

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw (SC'11): 10 rounds of two 32x32->64 multiplies per round with
// a Weyl key schedule.  Counter (pixel, sample, bounce, dim/4), key (lo32, hi32 of seed).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi_a = __umulhi(0xD2511F53u, c.x), lo_a = 0xD2511F53u * c.x;
        const uint32_t hi_b = __umulhi(0xCD9E8D57u, c.z), lo_b = 0xCD9E8D57u * c.z;
        c = make_uint4(hi_b ^ c.y ^ k0, lo_b, hi_a ^ c.w ^ k1, lo_a);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}
// 24 high bits of a word -> [0, 1), exact in FP32
__device__ __forceinline__ float u24(uint32_t w) { return (float)(w >> 8) * (1.0f / 16777216.0f); }

// uniforms of one path vertex: call j covers dims 4j..4j+3
struct VertexRng {
    uint32_t p, s, k, k0, k1;
    __device__ __forceinline__ uint4 block(uint32_t j) const {
        return philox4x32_10(make_uint4(p, s, k, j), k0, k1);
    }
};

enum { DIM_CAM_X = 0, DIM_CAM_Y = 1, DIM_LIGHT_PICK = 2, DIM_LIGHT_U = 3, DIM_LIGHT_V = 4,
       DIM_LOBE = 5, DIM_DIR_U = 6, DIM_DIR_V = 7, DIM_REFRACT = 8, DIM_RR = 9 };

__device__ __forceinline__ float uniform_at(uint32_t p, uint32_t s, uint32_t k, uint32_t dim,
                                            uint64_t seed) {
    uint4 w = philox4x32_10(make_uint4(p, s, k, dim >> 2), (uint32_t)seed, (uint32_t)(seed >> 32));
    uint32_t sel = (dim & 3u) == 0 ? w.x : ((dim & 3u) == 1 ? w.y : ((dim & 3u) == 2 ? w.z : w.w));
    return u24(sel);
}

// ------------------------------------------------------------------ materials
// Device copy of pt_openpbr; emission premultiplied by its luminance.
struct __align__(16) DMat {
    float3 base_color; float base_weight;
    float3 spec_color; float metalness;
    float3 trans_color; float spec_weight;
    float3 coat_color; float trans_weight;
    float3 emission; float coat_weight;
    float spec_rough, spec_ior, coat_rough, coat_ior;
    float diffuse_rough, thin_walled;   // thin_walled: 0 or 1
    float spec_aniso, spec_rot;         // specular_roughness_anisotropy, tangent rotation (turns)
    float fuzz_weight, pad0, pad1, pad2;   // colour and width live in the material's fuzz block
};

struct __align__(16) DQuad {
    float3 p0; float area;
    float3 e1; int two_sided;
    float3 e2; float pad0;
    float3 L; float pad1;
    float3 n; float pad2;
};

// ------------------------------------------------------------------ Fresnel
__device__ __forceinline__ float fresnel_dielectric(float ci, float eta) {
    ci = fminf(fmaxf(ci, 0.0f), 1.0f);
    const float s2t = (1.0f - ci * ci) / (eta * eta);
    if (s2t >= 1.0f) return 1.0f;
    const float ct = sqrtf(1.0f - s2t);
    const float rpar = (eta * ci - ct) / (eta * ci + ct);
    const float rper = (ci - eta * ct) / (ci + eta * ct);
    return 0.5f * (rpar * rpar + rper * rper);
}

// F82-tint metal Fresnel: Schlick from F0 minus b mu (1-mu)^6 with F(1/7) = tint Schlick(1/7)
__device__ __forceinline__ float f82_channel(float f0, float tint, float mu) {
    const float mu_bar = 1.0f / 7.0f;
    const float ob = 1.0f - mu_bar;
    const float ob2 = ob * ob, ob5 = ob2 * ob2 * ob, ob6 = ob5 * ob;
    const float om = 1.0f - mu;
    const float om2 = om * om, om5 = om2 * om2 * om, om6 = om5 * om;
    const float schlick = f0 + (1.0f - f0) * om5;
    const float schlick_bar = f0 + (1.0f - f0) * ob5;
    const float b = schlick_bar * (1.0f - tint) / (mu_bar * ob6);
    const float f = schlick - b * mu * om6;
    return fminf(fmaxf(f, 0.0f), 1.0f);
}
__device__ __forceinline__ float3 fresnel_f82(float3 f0, float3 tint, float mu) {
    mu = fminf(fmaxf(mu, 0.0f), 1.0f);
    return mk3(f82_channel(f0.x, tint.x, mu), f82_channel(f0.y, tint.y, mu), f82_channel(f0.z, tint.z, mu));
}

// ------------------------------------------------------------------ GGX
// Anisotropic GGX: width ax along the tangent (local x), ay along the bitangent (local y);
// ax = ay is the isotropic lobe.  D = 1 / (pi ax ay (hx^2/ax^2 + hy^2/ay^2 + hz^2)^2),
// evaluated as ax ay / (pi d^2) with d = hx^2 (ay/ax) + hy^2 (ax/ay) + hz^2 ax ay: the two
// ratios depend on the closure only, so inlined calls share them.
__device__ __forceinline__ float ggx_D(float3 h, float ax, float ay) {
    if (h.z <= 0.0f) return 0.0f;
    const float axy = ax * ay;
    const float d = h.x * h.x * (ay / ax) + h.y * h.y * (ax / ay) + axy * (h.z * h.z);
    return axy / (PT_PI_F * d * d);
}
__device__ __forceinline__ float ggx_lambda(float3 w, float ax, float ay) {
    const float c2 = w.z * w.z;
    if (c2 <= 0.0f) return __int_as_float(0x7f800000);
    const float sx = ax * w.x, sy = ay * w.y;
    const float x = (sx * sx + sy * sy) / c2;
    return x / (2.0f * (1.0f + sqrtf(1.0f + x)));
}
__device__ __forceinline__ float ggx_G1(float3 w, float ax, float ay) { return 1.0f / (1.0f + ggx_lambda(w, ax, ay)); }
__device__ __forceinline__ float ggx_G2(float3 wo, float3 wi, float ax, float ay) {
    return 1.0f / (1.0f + ggx_lambda(wo, ax, ay) + ggx_lambda(wi, ax, ay));
}
__device__ __forceinline__ float ggx_vndf_pdf(float3 wo, float3 h, float ax, float ay) {
    const float oh = dot3(wo, h);
    if (oh <= 0.0f || wo.z <= 0.0f) return 0.0f;
    return ggx_G1(wo, ax, ay) * oh * ggx_D(h, ax, ay) / wo.z;
}
// visible-normal sampling (Heitz 2018): stretch, sample the projected half disk, unstretch
__device__ __forceinline__ float3 ggx_vndf_sample(float3 wo, float ax, float ay, float u1, float u2) {
    const float3 vh = norm3(mk3(ax * wo.x, ay * wo.y, wo.z));
    const float lensq = vh.x * vh.x + vh.y * vh.y;
    const float3 t1 = lensq > 0.0f ? mk3(-vh.y, vh.x, 0.0f) * (1.0f / sqrtf(lensq)) : mk3(1.0f, 0.0f, 0.0f);
    const float3 t2 = cross3(vh, t1);
    const float r = sqrtf(u1);
    const float phi = 2.0f * PT_PI_F * u2;
    float sp, cp;
    sincosf(phi, &sp, &cp);
    const float p1 = r * cp;
    float p2 = r * sp;
    const float s = 0.5f * (1.0f + vh.z);
    p2 = (1.0f - s) * sqrtf(fmaxf(0.0f, 1.0f - p1 * p1)) + s * p2;
    const float3 nh = t1 * p1 + t2 * p2 + vh * sqrtf(fmaxf(0.0f, 1.0f - p1 * p1 - p2 * p2));
    return norm3(mk3(ax * nh.x, ay * nh.y, fmaxf(0.0f, nh.z)));
}
__device__ __forceinline__ float3 reflect3(float3 wo, float3 h) { return h * (2.0f * dot3(wo, h)) - wo; }
__device__ __forceinline__ bool refract3(float3 wo, float3 h, float eta, float3& wi) {
    const float ci = dot3(wo, h);
    const float s2t = (1.0f - ci * ci) / (eta * eta);
    if (s2t >= 1.0f) return false;
    const float ct = sqrtf(1.0f - s2t);
    wi = wo * (-1.0f / eta) + h * (ci / eta - ct);
    return true;
}

// ------------------------------------------------------------------ fuzz (sheen) lobe
// The Charlie distribution D = (2 + 1/a) sin(theta_m)^(1/a) / (2 pi) (Estevez & Kulla 2017)
// with its exact Smith masking: G1 = mu / A(mu), A(mu) = int <w, m>+ D(m) dm its projected
// area, so the height-correlated lobe is D(h) / (4 (A(mu_i) mu_o + A(mu_o) mu_i - mu_i mu_o)).
// A and the lobe's directional albedo E have no closed form: per material the library keeps
// a fuzz block of FUZZ_FLOATS floats -- fw, fc[3], a (= max(fuzz_roughness, 0.2)^2), 3 unused,
// then A as a Chebyshev series in x = 2 mu - 1 (FUZZ_A_TERMS) and E as one in
// x = 2 mu^(1/4) - 1 (FUZZ_E_TERMS; E behaves like mu log mu at grazing) -- computed by
// quadrature when the material table is made (pt_fuzz.cu).  Only materials with fuzz read it.
constexpr int FUZZ_HEAD = 8, FUZZ_A_TERMS = 16, FUZZ_E_TERMS = 32;
constexpr int FUZZ_FLOATS = FUZZ_HEAD + FUZZ_A_TERMS + FUZZ_E_TERMS;

// sum_k c[k] T_k(x) by Clenshaw's recurrence
template <int N>
__device__ __forceinline__ float cheb_eval(const float* __restrict__ c, float x) {
    float b1 = 0.0f, b2 = 0.0f;
#pragma unroll
    for (int k = N - 1; k >= 1; --k) {
        const float t = 2.0f * x * b1 - b2 + __ldg(c + k);
        b2 = b1;
        b1 = t;
    }
    return x * b1 - b2 + __ldg(c);
}
__device__ __forceinline__ float fuzz_area(const float* fz, float mu) {
    return cheb_eval<FUZZ_A_TERMS>(fz + FUZZ_HEAD, 2.0f * fminf(fmaxf(mu, 0.0f), 1.0f) - 1.0f);
}
__device__ __forceinline__ float fuzz_albedo(const float* fz, float mu) {
    return cheb_eval<FUZZ_E_TERMS>(fz + FUZZ_HEAD + FUZZ_A_TERMS,
                                   2.0f * sqrtf(sqrtf(fminf(fmaxf(mu, 0.0f), 1.0f))) - 1.0f);
}
__device__ __forceinline__ float sheen_D(float cos_m, float alpha) {
    const float s2 = fmaxf(0.0f, 1.0f - cos_m * cos_m);
    return (2.0f + 1.0f / alpha) * powf(s2, 0.5f / alpha) * (0.5f * PT_INV_PI_F);
}

// ------------------------------------------------------------------ OpenPBR closure
// f = fw fc f_fuzz + A_f (cw f_coat + A_c (m f_metal + (1 - m) f_diel)), lobes coat / metal /
// dielectric / diffuse / fuzz, picked with probability proportional to an albedo estimate at
// wo (one-sample MIS).  A_f = (1 - fw) + fw (1 - E(|mu_i|)) (1 - E(mu_o)).
enum { LOBE_COAT = 0, LOBE_METAL = 1, LOBE_DIEL = 2, LOBE_DIFF = 3, LOBE_FUZZ = 4, N_LOBES = 5 };

struct Closure {
    float3 bc, sc, tc, cc;
    float bw, m, sw, t, cw, dr;
    float eta_s, eta_c, ax_s, ay_s, a_c;   // specular widths along tangent / bitangent; coat
    bool delta_s, delta_c, any, has_smooth, thin;
    const float* fz;            // the material's fuzz block, nullptr without fuzz
    float fe_o, fa_o;           // with fuzz: E(mu_o), A(mu_o) of the setup's mu_o
    float p[N_LOBES];
};

// fz: the material's fuzz block (read only when its fuzz_weight is > 0).  FUZZ = false
// compiles the closure without the fuzz layer, for kernels that render scenes without it.
template <bool FUZZ = true>
__device__ __forceinline__ void closure_setup(Closure& C, const DMat& M, bool front, float mu_o, const float* fz) {
    C.bc = M.base_color; C.bw = M.base_weight; C.m = M.metalness; C.dr = M.diffuse_rough;
    C.sc = M.spec_color; C.sw = M.spec_weight;
    C.tc = M.trans_color; C.t = M.trans_weight;
    C.cc = M.coat_color; C.cw = M.coat_weight;
    C.thin = M.thin_walled != 0.0f;
    // a thin-walled sheet has the same medium on both sides
    C.eta_s = (C.t > 0.0f && !front && !C.thin) ? 1.0f / M.spec_ior : M.spec_ior;
    C.eta_c = M.coat_ior;
    // OpenPBR's anisotropy mapping: ax = r^2 sqrt(2 / (1 + (1-a)^2)), ay = (1-a) ax (a = 0:
    // both r^2); a delta lobe when ax < 1e-4, else the narrower width is kept >= 1e-4
    const float r2 = M.spec_rough * M.spec_rough, ia = 1.0f - M.spec_aniso;
    const float at = r2 * sqrtf(2.0f / (1.0f + ia * ia));
    C.ax_s = at;
    C.ay_s = fmaxf(ia * at, 1e-4f);
    C.a_c = M.coat_rough * M.coat_rough;
    C.delta_s = at < 1e-4f;
    C.delta_c = C.a_c < 1e-4f;
    const float fc = fresnel_dielectric(mu_o, C.eta_c);
    const float w_coat = C.cw * fc;
    const float att = C.cw * lum3(C.cc) * (1.0f - fc) + (1.0f - C.cw);
    const float3 f0 = C.bc * C.bw;
    const float w_metal = att * C.m * C.sw * lum3(fresnel_f82(f0, C.sc, mu_o));
    const float fs = fresnel_dielectric(mu_o, C.eta_s);
    const float w_spec = att * (1.0f - C.m) * C.sw * lum3(C.sc) * fs;
    const float w_trans = att * (1.0f - C.m) * C.t * lum3(C.tc) * (1.0f - C.sw * fs);
    float w_diff = att * (1.0f - C.m) * (1.0f - C.t) * (1.0f - C.sw * fs) * lum3(f0);
    float w2 = w_spec + w_trans, wc = w_coat, wm = w_metal, w_fuzz = 0.0f;
    C.fz = nullptr;
    if (FUZZ && M.fuzz_weight > 0.0f) {
        C.fz = fz;
        const float fw = M.fuzz_weight, e_o = fuzz_albedo(fz, mu_o);
        C.fe_o = e_o;
        C.fa_o = fuzz_area(fz, mu_o);
        const float sc = 1.0f - fw * e_o;
        wc *= sc; wm *= sc; w2 *= sc; w_diff *= sc;
        w_fuzz = fw * lum3(mk3(__ldg(fz + 1), __ldg(fz + 2), __ldg(fz + 3))) * e_o;
    }
    const float sum = wc + wm + w2 + w_diff + w_fuzz;
    C.any = sum > 0.0f;
    const float inv = C.any ? 1.0f / sum : 0.0f;
    C.p[0] = wc * inv; C.p[1] = wm * inv; C.p[2] = w2 * inv; C.p[3] = w_diff * inv; C.p[4] = FUZZ ? w_fuzz * inv : 0.0f;
    C.has_smooth = (C.p[0] > 0.0f && !C.delta_c) || ((C.p[1] > 0.0f || C.p[2] > 0.0f) && !C.delta_s) ||
                   C.p[3] > 0.0f || C.p[4] > 0.0f;
}

// A_f: the part of the layers under the fuzz that reaches wo from wi (1 without fuzz); wo is
// the direction the closure was set up for
__device__ __forceinline__ float fuzz_attenuation(const Closure& C, float mi_abs) {
    if (C.fz == nullptr) return 1.0f;
    const float fw = __ldg(C.fz);
    return (1.0f - fw) + fw * (1.0f - fuzz_albedo(C.fz, mi_abs)) * (1.0f - C.fe_o);
}

__device__ __forceinline__ float diel_reflect_prob(const Closure& C, float F) {
    const float r = C.sw * lum3(C.sc) * F;
    const float t = C.t * lum3(C.tc) * (1.0f - C.sw * F);
    if (F >= 1.0f) return 1.0f;
    const float s = r + t;
    return s > 0.0f ? r / s : 1.0f;
}

__device__ __forceinline__ float3 coat_attenuation(const Closure& C, float mi_abs, float mo) {
    const float fci = fresnel_dielectric(mi_abs, C.eta_c);
    const float fco = fresnel_dielectric(mo, C.eta_c);
    return C.cc * (C.cw * (1.0f - fci) * (1.0f - fco)) + splat3(1.0f - C.cw);
}

// non-delta part of f(wo, wi) and the mixture pdf of sampling wi
__device__ __forceinline__ void closure_eval(const Closure& C, float3 wo, float3 wi, float3& f_out, float& pdf_out) {
    float3 f = splat3(0.0f);
    float pdf = 0.0f;
    f_out = f;
    pdf_out = 0.0f;
    const float mo = wo.z, mi = wi.z;
    if (mo <= 0.0f || mi == 0.0f) return;
    const float3 ac = coat_attenuation(C, fabsf(mi), mo);
    if (mi > 0.0f) {
        const float3 h = norm3(wo + wi);
        const float oh = dot3(wo, h);
        if (oh <= 0.0f) return;
        if (!C.delta_c && C.cw > 0.0f) {
            const float fr = fresnel_dielectric(oh, C.eta_c);
            const float val = C.cw * fr * ggx_D(h, C.a_c, C.a_c) * ggx_G2(wo, wi, C.a_c, C.a_c) / (4.0f * mo * mi);
            f = f + splat3(val);
            pdf += C.p[0] * ggx_vndf_pdf(wo, h, C.a_c, C.a_c) / (4.0f * oh);
        }
        if (!C.delta_s) {
            const float dg = ggx_D(h, C.ax_s, C.ay_s) * ggx_G2(wo, wi, C.ax_s, C.ay_s) / (4.0f * mo * mi);
            const float vndf = ggx_vndf_pdf(wo, h, C.ax_s, C.ay_s) / (4.0f * oh);
            if (C.m > 0.0f) {
                const float3 fm = fresnel_f82(C.bc * C.bw, C.sc, oh);
                f = f + (ac * fm) * (C.m * C.sw * dg);
            }
            pdf += C.p[1] * vndf;
            const float fr = fresnel_dielectric(oh, C.eta_s);
            f = f + (ac * C.sc) * ((1.0f - C.m) * C.sw * fr * dg);
            pdf += C.p[2] * diel_reflect_prob(C, fr) * vndf;
        }
        const float fsi = fresnel_dielectric(mi, C.eta_s);
        const float fso = fresnel_dielectric(mo, C.eta_s);
        float kd = (1.0f - C.m) * (1.0f - C.t) * (1.0f - C.sw * fsi) * (1.0f - C.sw * fso) * C.bw * PT_INV_PI_F;
        if (C.dr > 0.0f) {
            // rough diffuse base: qualitative Oren-Nayar factor (1 + sigma s/t) / (1 + c sigma),
            // c = 1/2 - 2/(3 pi), s = wi.wo - mu_i mu_o, t = max(mu_i, mu_o) if s > 0 else 1
            const float s = dot3(wo, wi) - mo * mi;
            const float t = s > 0.0f ? fmaxf(mo, mi) : 1.0f;
            kd *= (1.0f + C.dr * s / t) / (1.0f + 0.287793409f * C.dr);
        }
        f = f + (ac * C.bc) * kd;
        pdf += C.p[3] * mi * PT_INV_PI_F;
    } else if (C.thin) {
        // thin-walled transmission: the reflection lobe mirrored through the surface plane
        if (!C.delta_s && C.t > 0.0f) {
            const float3 wm = mk3(wi.x, wi.y, -wi.z);
            const float3 h = norm3(wo + wm);
            const float oh = dot3(wo, h);
            if (oh > 0.0f) {
                const float fr = fresnel_dielectric(oh, C.eta_s);
                const float dg = ggx_D(h, C.ax_s, C.ay_s) * ggx_G2(wo, wm, C.ax_s, C.ay_s) / (4.0f * mo * fabsf(mi));
                const float val = (1.0f - C.m) * C.t * (1.0f - C.sw * fr) * dg;
                f = f + (ac * C.tc) * val;
                pdf += C.p[2] * (1.0f - diel_reflect_prob(C, fr)) * ggx_vndf_pdf(wo, h, C.ax_s, C.ay_s) / (4.0f * oh);
            }
        }
    } else if (!C.delta_s && C.t > 0.0f) {
        const float eta = C.eta_s;
        float3 h = norm3(wo + wi * eta);
        if (h.z < 0.0f) h = -h;
        const float oh = dot3(wo, h), ih = dot3(wi, h);
        if (oh > 0.0f && ih < 0.0f) {
            const float fr = fresnel_dielectric(oh, eta);
            const float denom = oh + eta * ih;
            const float dg = ggx_D(h, C.ax_s, C.ay_s) * ggx_G2(wo, wi, C.ax_s, C.ay_s);
            const float val = (1.0f - C.m) * C.t * (1.0f - C.sw * fr) * dg * fabsf(ih) * oh /
                              (fabsf(mi) * mo * denom * denom);
            f = f + (ac * C.tc) * val;
            pdf += C.p[2] * (1.0f - diel_reflect_prob(C, fr)) * ggx_vndf_pdf(wo, h, C.ax_s, C.ay_s) * eta * eta *
                   fabsf(ih) / (denom * denom);
        }
    }
    if (C.fz != nullptr) {
        f = f * fuzz_attenuation(C, fabsf(mi));
        if (mi > 0.0f) {
            const float* fz = C.fz;
            const float3 h = norm3(wo + wi);
            const float den = 4.0f * (fuzz_area(fz, mi) * mo + C.fa_o * mi - mi * mo);
            const float3 fc = mk3(__ldg(fz + 1), __ldg(fz + 2), __ldg(fz + 3));
            f = f + fc * (__ldg(fz) * sheen_D(h.z, __ldg(fz + 4)) / den);
            pdf += C.p[LOBE_FUZZ] * (0.5f * PT_INV_PI_F);
        }
    }
    f_out = f;
    pdf_out = pdf;
}

struct BsdfSample {
    float3 wi;
    float3 weight;
    float pdf;
    bool delta;
};

__device__ __forceinline__ bool closure_sample(const Closure& C, float3 wo, float u_lobe, float u1, float u2,
                                               float u_refr, BsdfSample& out) {
    if (!C.any || wo.z <= 0.0f) return false;
    int lobe = -1, last = -1;
    float c = 0.0f;
#pragma unroll
    for (int j = 0; j < N_LOBES; ++j) {
        if (C.p[j] > 0.0f && lobe < 0) {
            last = j;
            c += C.p[j];
            if (u_lobe < c) lobe = j;
        }
    }
    if (lobe < 0) lobe = last;
    const float mo = wo.z;
    float3 wi;
    out.delta = false;
    out.pdf = 0.0f;
    if (lobe == LOBE_COAT) {
        if (C.delta_c) {
            out.wi = mk3(-wo.x, -wo.y, wo.z);
            out.weight = splat3(C.cw * fresnel_dielectric(mo, C.eta_c) * fuzz_attenuation(C, mo) / C.p[0]);
            out.delta = true;
            return true;
        }
        wi = reflect3(wo, ggx_vndf_sample(wo, C.a_c, C.a_c, u1, u2));
        if (wi.z <= 0.0f) return false;
    } else if (lobe == LOBE_METAL) {
        if (C.delta_s) {
            out.wi = mk3(-wo.x, -wo.y, wo.z);
            const float3 fm = fresnel_f82(C.bc * C.bw, C.sc, mo);
            out.weight = (coat_attenuation(C, mo, mo) * fm) * (C.m * C.sw * fuzz_attenuation(C, mo) / C.p[1]);
            out.delta = true;
            return true;
        }
        wi = reflect3(wo, ggx_vndf_sample(wo, C.ax_s, C.ay_s, u1, u2));
        if (wi.z <= 0.0f) return false;
    } else if (lobe == LOBE_DIEL) {
        const float3 h = C.delta_s ? mk3(0.0f, 0.0f, 1.0f) : ggx_vndf_sample(wo, C.ax_s, C.ay_s, u1, u2);
        const float oh = dot3(wo, h);
        if (oh <= 0.0f) return false;
        const float fr = fresnel_dielectric(oh, C.eta_s);
        const float pr = diel_reflect_prob(C, fr);
        const bool do_reflect = u_refr < pr;
        if (do_reflect) {
            wi = reflect3(wo, h);
            if (wi.z <= 0.0f) return false;
        } else if (C.thin) {
            // the reflected direction mirrored through the surface plane
            const float3 wr = reflect3(wo, h);
            if (wr.z <= 0.0f) return false;
            wi = mk3(wr.x, wr.y, -wr.z);
        } else {
            if (!refract3(wo, h, C.eta_s, wi)) return false;
            if (wi.z >= 0.0f) return false;
        }
        if (C.delta_s) {
            out.wi = wi;
            out.delta = true;
            if (do_reflect) {
                out.weight = (coat_attenuation(C, mo, mo) * C.sc) *
                             ((1.0f - C.m) * C.sw * fr * fuzz_attenuation(C, mo) / (C.p[2] * pr));
            } else {
                const float scale = C.thin ? 1.0f : C.eta_s * C.eta_s;   // radiance across the interface
                out.weight = (coat_attenuation(C, fabsf(wi.z), mo) * C.tc) *
                             ((1.0f - C.m) * C.t * (1.0f - C.sw * fr) * fuzz_attenuation(C, fabsf(wi.z)) /
                              (scale * C.p[2] * (1.0f - pr)));
            }
            return true;
        }
    } else if (lobe == LOBE_DIFF) {
        const float r = sqrtf(u1), phi = 2.0f * PT_PI_F * u2;
        float sp, cp;
        sincosf(phi, &sp, &cp);
        wi = mk3(r * cp, r * sp, sqrtf(fmaxf(0.0f, 1.0f - u1)));
        if (wi.z <= 0.0f) return false;
    } else {
        // fuzz: uniform over the upper hemisphere
        const float r = sqrtf(fmaxf(0.0f, 1.0f - u1 * u1)), phi = 2.0f * PT_PI_F * u2;
        float sp, cp;
        sincosf(phi, &sp, &cp);
        wi = mk3(r * cp, r * sp, u1);
        if (wi.z <= 0.0f) return false;
    }
    float3 f;
    float pdf;
    closure_eval(C, wo, wi, f, pdf);
    if (!(pdf > 0.0f)) return false;
    out.wi = wi;
    out.pdf = pdf;
    out.weight = f * (fabsf(wi.z) / pdf);
    return true;
}

// orthonormal basis around n (Duff et al. 2017)
__device__ __forceinline__ void onb(float3 n, float3& t, float3& b) {
    const float s = n.z >= 0.0f ? 1.0f : -1.0f;
    const float a = -1.0f / (s + n.z);
    const float c = n.x * n.y * a;
    t = mk3(1.0f + s * n.x * n.x * a, s * c, -s * n.x);
    b = mk3(c, s + n.y * n.y * a, -n.y);
}

// Frame of an anisotropic surface: the interface carries no vertex tangents, so the tangent
// is the triangle's first edge e1 projected into the shading plane, t0 = normalize(e1 -
// n (n.e1)), turned about n by `rot` turns: t = cos(2 pi rot) t0 + sin(2 pi rot) (n x t0),
// b = n x t; (t, b, n) is right-handed.
__device__ __forceinline__ void tangent_frame(float3 n, float3 e1, float rot, float3& t, float3& b) {
    const float3 p = e1 - n * dot3(n, e1);
    const float l2 = dot3(p, p);
    if (!(l2 > 0.0f)) { onb(n, t, b); return; }
    const float3 t0 = p * (1.0f / sqrtf(l2));
    const float3 b0 = cross3(n, t0);
    float sr, cr;
    sincospif(2.0f * rot, &sr, &cr);
    t = t0 * cr + b0 * sr;
    b = cross3(n, t);
}

__device__ __forceinline__ float power_heuristic(float pa, float pb) {
    const float a2 = pa * pa, b2 = pb * pb;
    return a2 + b2 > 0.0f ? a2 / (a2 + b2) : 0.0f;
}

// ------------------------------------------------------------------ scene on the device
// Triangle record (48 B, three float4): v0.xyz + original triangle id (bits),
// v1.xyz + material code (material id, or 0x80000000 | light index), v2.xyz + unused.
#define PT_LIGHT_BIT 0x80000000u
#define PT_NO_HIT 0xFFFFFFFFu
#define PT_STACK 96

struct DScene {
    const float4* tris;        // leaf order
    const uint4* nodes;        // compressed 8-wide BVH, 5 x uint4 per node
    const DMat* mats;
    const float* fuzz;         // FUZZ_FLOATS per material: the fuzz lobe's series
    const DQuad* quads;
    const float* env;          // env_h * env_w * 3
    const float* env_marg;     // env_h + 1
    const float* env_cond;     // env_h * (env_w + 1)
    const float* env_wtex;     // env_h * env_w (unnormalised weights)
    const int* env_guide;      // search guides: env_gm + 1 for the marginal, then env_gc + 1 per row
    uint32_t* err;             // sticky error bits
    float env_total;
    float eps;
    int env_w, env_h;
    int n_quads;
    int n_nodes;
    int n_tris;
    int env_gm, env_gc;        // guide sizes (powers of two)
    int pad;
};

// ---- watertight ray/triangle test (Woop, Benthin, Wald, JCGT 2(1), 2013) ----
struct WRay {
    float3 o;
    int kx, ky, kz;
    float sx, sy, sz;
};

__device__ __forceinline__ WRay make_wray(float3 o, float3 d) {
    WRay r;
    r.o = o;
    const float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    int kz = 0;
    float m = ax;
    if (ay > m) { kz = 1; m = ay; }
    if (az > m) { kz = 2; }
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    if (comp3(d, kz) < 0.0f) { const int t = kx; kx = ky; ky = t; }
    r.kx = kx; r.ky = ky; r.kz = kz;
    const float dz = comp3(d, kz);
    r.sx = __fdiv_rn(comp3(d, kx), dz);
    r.sy = __fdiv_rn(comp3(d, ky), dz);
    r.sz = __fdiv_rn(1.0f, dz);
    return r;
}

// Edge functions use explicitly rounded products and differences (no FMA contraction) so
// that two triangles sharing an edge evaluate exactly opposite values: no ray leaks.
__device__ __forceinline__ bool tri_hit(const WRay& r, float3 p0, float3 p1, float3 p2, float tmax,
                                        float& t_out, float& u_out, float& v_out) {
    const float3 A = mk3(__fsub_rn(p0.x, r.o.x), __fsub_rn(p0.y, r.o.y), __fsub_rn(p0.z, r.o.z));
    const float3 B = mk3(__fsub_rn(p1.x, r.o.x), __fsub_rn(p1.y, r.o.y), __fsub_rn(p1.z, r.o.z));
    const float3 Cc = mk3(__fsub_rn(p2.x, r.o.x), __fsub_rn(p2.y, r.o.y), __fsub_rn(p2.z, r.o.z));
    const float Az = comp3(A, r.kz), Bz = comp3(B, r.kz), Cz = comp3(Cc, r.kz);
    const float ax = __fsub_rn(comp3(A, r.kx), __fmul_rn(r.sx, Az));
    const float ay = __fsub_rn(comp3(A, r.ky), __fmul_rn(r.sy, Az));
    const float bx = __fsub_rn(comp3(B, r.kx), __fmul_rn(r.sx, Bz));
    const float by = __fsub_rn(comp3(B, r.ky), __fmul_rn(r.sy, Bz));
    const float cx = __fsub_rn(comp3(Cc, r.kx), __fmul_rn(r.sx, Cz));
    const float cy = __fsub_rn(comp3(Cc, r.ky), __fmul_rn(r.sy, Cz));
    const float U = __fsub_rn(__fmul_rn(cx, by), __fmul_rn(cy, bx));
    const float V = __fsub_rn(__fmul_rn(ax, cy), __fmul_rn(ay, cx));
    const float W = __fsub_rn(__fmul_rn(bx, ay), __fmul_rn(by, ax));
    if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return false;
    const float det = U + V + W;
    if (det == 0.0f) return false;
    const float T = U * (r.sz * Az) + V * (r.sz * Bz) + W * (r.sz * Cz);
    const float t = __fdiv_rn(T, det);
    if (!(t > 0.0f) || !(t < tmax)) return false;
    t_out = t;
    u_out = __fdiv_rn(V, det);
    v_out = __fdiv_rn(W, det);
    return true;
}

// ---- compressed 8-wide BVH node (80 B) ----
// n0 = p.xyz (float bits), w = ex | ey<<8 | ez<<16 | imask<<24
// n1 = child_base, tri_base, meta[0..3], meta[4..7]
// n2..n4 = qlo_x, qlo_y, qlo_z, qhi_x, qhi_y, qhi_z (8 bytes each)
// meta: 0 = empty slot; internal child: nonzero, node = child_base + rank among internal
// slots; leaf child: count << 5 | offset, triangles tri_base + offset .. + count.
__device__ __forceinline__ uint32_t byte_of(uint32_t lo4, uint32_t hi4, int i) {
    return ((i < 4 ? lo4 : hi4) >> (8 * (i & 3))) & 0xffu;
}

struct TravRay {
    float3 o, d, inv;
};
__device__ __forceinline__ TravRay make_trav(float3 o, float3 d) {
    TravRay r;
    r.o = o;
    r.d = d;
    const float big = 1e20f;
    r.inv = mk3(fabsf(d.x) > 1e-20f ? 1.0f / d.x : copysignf(big, d.x),
                fabsf(d.y) > 1e-20f ? 1.0f / d.y : copysignf(big, d.y),
                fabsf(d.z) > 1e-20f ? 1.0f / d.z : copysignf(big, d.z));
    return r;
}

struct NodeView {
    float3 p, scale;
    uint32_t imask, child_base, tri_base, meta_lo, meta_hi;
    uint4 q0, q1, q2;
};

__device__ __forceinline__ NodeView load_node(const uint4* __restrict__ nodes, uint32_t i) {
    const uint4* b = nodes + 5u * i;
    const uint4 n0 = __ldg(b + 0), n1 = __ldg(b + 1);
    NodeView v;
    v.q0 = __ldg(b + 2);
    v.q1 = __ldg(b + 3);
    v.q2 = __ldg(b + 4);
    v.p = mk3(__uint_as_float(n0.x), __uint_as_float(n0.y), __uint_as_float(n0.z));
    v.scale = mk3(__uint_as_float((n0.w & 0xffu) << 23), __uint_as_float(((n0.w >> 8) & 0xffu) << 23),
                  __uint_as_float(((n0.w >> 16) & 0xffu) << 23));
    v.imask = n0.w >> 24;
    v.child_base = n1.x;
    v.tri_base = n1.y;
    v.meta_lo = n1.z;
    v.meta_hi = n1.w;
    return v;
}

// Per-node setup of the child box tests.  Along each axis the near and far planes of child
// slot i are p + q_near(i) * scale and p + q_far(i) * scale (near/far chosen once per ray by
// the direction's sign), so their ray distances are q * b + (p - o)/d with b = scale/d.  The
// byte q is read as the float f = 1 + q / 2^15 (the byte placed in the mantissa of 1.0, no
// conversion instruction), and the distance is evaluated as fma(f, B, c) with B = 2^15 b
// (exact: a power of two times b) and c = (p - o)/d - B (one more rounding).  eps widens
// every slab by a bound on the rounding of those terms: the subtraction, the products and
// the fma (at most 4 units of the last place of |(p - o)/d| + 255 |b|), the builder's
// one-rounding decode of the plane (|p/d| + 255 |b|) and the rounding of c (half a unit of
// the last place of 2^15 |b|, i.e. at most 2^-9 |b|): 4e-7 (|(p - o)/d| + 255 |b| + |p/d|) +
// 4e-3 |b| covers them, so the test stays conservative.  (A B or c that overflows makes that
// axis's distances NaN, which fmaxf/fminf ignore: the box is then tested on the other axes
// only, which is conservative too.)
struct NodeTest {
    float3 cn, cf, B;                              // (p - o)/d -/+ eps - B, B = 2^15 scale/d
    uint32_t nx0, nx1, ny0, ny1, nz0, nz1;         // near-plane byte words per axis
    uint32_t fx0, fx1, fy0, fy1, fz0, fz1;         // far-plane byte words per axis
};

// byte i of the 8-byte array (w0, w1) in bits 8..15 of 1.0f: the float 1 + q / 2^15, exactly
__device__ __forceinline__ float qbyte(uint32_t w0, uint32_t w1, int i) {
    return __uint_as_float(__byte_perm(i < 4 ? w0 : w1, 0x3F800000u, 0x7604u | ((uint32_t)(i & 3) << 4)));
}

__device__ __forceinline__ void node_setup(const NodeView& v, const TravRay& r, NodeTest& T) {
    const float ax = __fmul_rn(__fsub_rn(v.p.x, r.o.x), r.inv.x);
    const float ay = __fmul_rn(__fsub_rn(v.p.y, r.o.y), r.inv.y);
    const float az = __fmul_rn(__fsub_rn(v.p.z, r.o.z), r.inv.z);
    const float bx = v.scale.x * r.inv.x, by = v.scale.y * r.inv.y, bz = v.scale.z * r.inv.z;
    T.B = mk3(bx * 32768.0f, by * 32768.0f, bz * 32768.0f);
    const float ex = 4e-7f * (fabsf(ax) + 10240.0f * fabsf(bx) + fabsf(v.p.x * r.inv.x));
    const float ey = 4e-7f * (fabsf(ay) + 10240.0f * fabsf(by) + fabsf(v.p.y * r.inv.y));
    const float ez = 4e-7f * (fabsf(az) + 10240.0f * fabsf(bz) + fabsf(v.p.z * r.inv.z));
    T.cn = mk3((ax - ex) - T.B.x, (ay - ey) - T.B.y, (az - ez) - T.B.z);
    T.cf = mk3((ax + ex) - T.B.x, (ay + ey) - T.B.y, (az + ez) - T.B.z);
    const bool px = r.inv.x >= 0.0f, py = r.inv.y >= 0.0f, pz = r.inv.z >= 0.0f;
    // lo words: x (q0.x, q0.y), y (q0.z, q0.w), z (q1.x, q1.y); hi: x (q1.z, q1.w), y (q2.x, q2.y), z (q2.z, q2.w)
    T.nx0 = px ? v.q0.x : v.q1.z; T.nx1 = px ? v.q0.y : v.q1.w;
    T.fx0 = px ? v.q1.z : v.q0.x; T.fx1 = px ? v.q1.w : v.q0.y;
    T.ny0 = py ? v.q0.z : v.q2.x; T.ny1 = py ? v.q0.w : v.q2.y;
    T.fy0 = py ? v.q2.x : v.q0.z; T.fy1 = py ? v.q2.y : v.q0.w;
    T.nz0 = pz ? v.q1.x : v.q2.z; T.nz1 = pz ? v.q1.y : v.q2.w;
    T.fz0 = pz ? v.q2.z : v.q1.x; T.fz1 = pz ? v.q2.w : v.q1.y;
}

// entry distance of child slot i, or -1 if the ray misses its box within [0, tmax]
__device__ __forceinline__ float child_test(const NodeTest& T, int i, float tmax) {
    const float ex = fmaf(qbyte(T.nx0, T.nx1, i), T.B.x, T.cn.x);
    const float ey = fmaf(qbyte(T.ny0, T.ny1, i), T.B.y, T.cn.y);
    const float ez = fmaf(qbyte(T.nz0, T.nz1, i), T.B.z, T.cn.z);
    const float xx = fmaf(qbyte(T.fx0, T.fx1, i), T.B.x, T.cf.x);
    const float xy = fmaf(qbyte(T.fy0, T.fy1, i), T.B.y, T.cf.y);
    const float xz = fmaf(qbyte(T.fz0, T.fz1, i), T.B.z, T.cf.z);
    const float tn = fmaxf(fmaxf(ex, ey), fmaxf(ez, 0.0f));
    const float tf = fminf(fminf(xx, xy), fminf(xz, tmax));
    return tn <= tf ? tn : -1.0f;
}

struct HitRec {
    float t, u, v;
    uint32_t tri;   // index into the leaf-ordered triangle array, PT_NO_HIT on a miss
};

// Node visits and triangle tests of one traversal (counting variant only).
struct TravCount {
    uint32_t nodes, tris, boxes;   // node visits, triangle tests, child box tests (filled slots)
};

// child slots of a node that hold a child (nonzero meta bytes): the box tests of one visit
__device__ __forceinline__ uint32_t node_slots(const NodeView& v) {
    return (uint32_t)(__popc(__vcmpne4(v.meta_lo, 0u)) + __popc(__vcmpne4(v.meta_hi, 0u))) >> 3;
}

// Closest-hit traversal as a state machine: closest_init sets up one ray, closest_step
// processes one node (eight unrolled box tests; the nearest internal child is descended
// into, the others go on the stack; leaf children are collected in a bit mask and their
// triangles intersected afterwards by one loop, so the triangle test exists once in the
// code) and returns true once the ray is finished; trace_closest_t runs one ray to
// completion.  (Refilling a finished lane with a new ray between steps was measured slower
// on the 1080p CAD frame: lanes at different depths diverge more than idle lanes cost.)
// Equal t resolves towards the lower original triangle id.
struct ClosestState {
    WRay wr;
    TravRay tr;
    float tmax;
    HitRec h;
    uint32_t best_orig, node, budget;
    int sp;
};

__device__ __forceinline__ void closest_init(const DScene& S, float3 o, float3 d, float tmax, ClosestState& st) {
    st.wr = make_wray(o, d);
    st.tr = make_trav(o, d);
    st.tmax = tmax;
    st.h.t = tmax;
    st.h.tri = PT_NO_HIT;
    st.h.u = st.h.v = 0.0f;
    st.best_orig = PT_NO_HIT;
    st.node = 0;
    st.sp = 0;
    // a tree traversal visits every node at most once: more visits mean a malformed tree
    st.budget = (uint32_t)S.n_nodes + 1u;
}

// The stack is a separate local array so the scalar state stays in registers.  It has
// PT_STACK_SLACK spare entries: a node's child loop writes its pushes without a capacity
// check inside the loop (at most 7 a node, so no write leaves the array) and the overflow of
// the PT_STACK entries the traversal may use is checked once after it.
// BRANCHLESS selects the form of the child loop; both push the same children in the same
// order.  The per-bounce closest-hit kernel keeps the branching form (a slot that misses
// skips the push logic): on the 1080p CAD frame it measured 3.68 against 3.99 ms a step.  The
// out-of-line traversal that the tail kernel and the megakernel call takes the form without
// branches, which measured faster there (tail kernel 0.49 -> 0.41 ms a step on the same
// frame, 1.45 -> 1.19 ms on the 5.2M-triangle scene), where the lanes of a warp are at
// different bounces and stages.
#define PT_STACK_SLACK 7
template <bool COUNT, bool BRANCHLESS = false>
__device__ __forceinline__ bool closest_step(const DScene& S, ClosestState& st, uint2 (&stack)[PT_STACK + PT_STACK_SLACK],
                                             TravCount& tc) {
    if (S.n_nodes == 0) return true;
    if (st.budget-- == 0u) { atomicOr(S.err, 4u); st.h.tri = PT_NO_HIT; return true; }
    const NodeView v = load_node(S.nodes, st.node);
    if (COUNT) { tc.nodes++; tc.boxes += node_slots(v); }
    NodeTest T;
    node_setup(v, st.tr, T);
    uint32_t leafmask = 0u;
    uint32_t near_node = PT_NO_HIT;
    float near_t = __int_as_float(0x7f800000);
    // the slots in order: a hit internal child nearer than the nearest so far displaces it
    // onto the stack, else goes there itself; a hit leaf joins the mask
    if constexpr (BRANCHLESS) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float tn = child_test(T, i, st.h.t);   // tn <= h.t whenever it is >= 0
            const bool hit = byte_of(v.meta_lo, v.meta_hi, i) != 0u && tn >= 0.0f;
            const bool inner = (v.imask >> i) & 1u;
            leafmask |= (hit && !inner) ? (1u << i) : 0u;
            const bool ih = hit && inner;
            const uint32_t c = v.child_base + __popc(v.imask & ((1u << i) - 1u));
            const bool nearer = ih && tn < near_t;
            const uint32_t push_node = nearer ? near_node : c;
            const float push_t = nearer ? near_t : tn;
            near_node = nearer ? c : near_node;
            near_t = nearer ? tn : near_t;
            if (ih && push_node != PT_NO_HIT) stack[st.sp++] = make_uint2(push_node, __float_as_uint(push_t));
        }
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (byte_of(v.meta_lo, v.meta_hi, i) == 0u) continue;
            const float tn = child_test(T, i, st.h.t);
            if (!(tn >= 0.0f && tn <= st.h.t)) continue;
            if ((v.imask >> i) & 1u) {
                const uint32_t c = v.child_base + __popc(v.imask & ((1u << i) - 1u));
                uint32_t push_node = c;
                float push_t = tn;
                if (tn < near_t) {
                    push_node = near_node;
                    push_t = near_t;
                    near_node = c;
                    near_t = tn;
                }
                if (push_node != PT_NO_HIT) stack[st.sp++] = make_uint2(push_node, __float_as_uint(push_t));
            } else {
                leafmask |= 1u << i;
            }
        }
    }
    if (st.sp > PT_STACK) { atomicOr(S.err, 1u); return true; }
    while (leafmask) {
        const int i = __ffs(leafmask) - 1;
        leafmask &= leafmask - 1u;
        const uint32_t meta = byte_of(v.meta_lo, v.meta_hi, i);
        const uint32_t first = v.tri_base + (meta & 31u);
        const uint32_t cnt = meta >> 5;
        if (COUNT) tc.tris += cnt;
        for (uint32_t k = 0; k < cnt; ++k) {
            const uint32_t ti = first + k;
            const float4 a = __ldg(S.tris + 3u * ti), b = __ldg(S.tris + 3u * ti + 1), c = __ldg(S.tris + 3u * ti + 2);
            float t, u, w;
            if (tri_hit(st.wr, xyz(a), xyz(b), xyz(c), st.tmax, t, u, w)) {
                const uint32_t orig = __float_as_uint(a.w);
                if (t < st.h.t || (t == st.h.t && orig < st.best_orig)) {
                    st.h.t = t; st.h.u = u; st.h.v = w; st.h.tri = ti; st.best_orig = orig;
                }
            }
        }
    }
    if (near_node != PT_NO_HIT && near_t <= st.h.t) {
        st.node = near_node;
        return false;
    }
    // pop the next child whose entry distance is still within the closest hit
    while (st.sp > 0) {
        const uint2 e = stack[--st.sp];
        if (__uint_as_float(e.y) <= st.h.t) { st.node = e.x; return false; }
    }
    return true;
}

template <bool COUNT, bool BRANCHLESS = false>
__device__ __forceinline__ void trace_closest_t(const DScene& S, float3 o, float3 d, float tmax, HitRec& h,
                                                TravCount& tc) {
    ClosestState st;
    uint2 stack[PT_STACK + PT_STACK_SLACK];
    closest_init(S, o, d, tmax, st);
    while (!closest_step<COUNT, BRANCHLESS>(S, st, stack, tc)) {
    }
    h = st.h;
}

// Any hit in (0, tmax): occlusion test for shadow rays, in the same step form.
struct AnyState {
    WRay wr;
    TravRay tr;
    float tmax;
    uint32_t node, budget;
    int sp;
    bool hit;
};

__device__ __forceinline__ void any_init(const DScene& S, float3 o, float3 d, float tmax, AnyState& st) {
    st.wr = make_wray(o, d);
    st.tr = make_trav(o, d);
    st.tmax = tmax;
    st.node = 0;
    st.sp = 0;
    st.hit = false;
    st.budget = (uint32_t)S.n_nodes + 1u;
}

template <bool COUNT>
__device__ __forceinline__ bool any_step(const DScene& S, AnyState& st, uint32_t (&stack)[PT_STACK + PT_STACK_SLACK],
                                         TravCount& tc) {
    if (S.n_nodes == 0) return true;
    if (st.budget-- == 0u) { atomicOr(S.err, 4u); return true; }
    const NodeView v = load_node(S.nodes, st.node);
    if (COUNT) { tc.nodes++; tc.boxes += node_slots(v); }
    NodeTest T;
    node_setup(v, st.tr, T);
    uint32_t leafmask = 0u;
    uint32_t next = PT_NO_HIT;
    // the first hit internal child is descended into, the later ones pushed; written without
    // branches (shadow pass 1.91 -> 1.88 ms a step on the 1080p CAD frame, 1.49 -> 1.39 ms on
    // the 5.2M-triangle scene, against a loop that skips the push logic of missed slots)
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float tn = child_test(T, i, st.tmax);
        const bool hit = byte_of(v.meta_lo, v.meta_hi, i) != 0u && tn >= 0.0f;
        const bool inner = (v.imask >> i) & 1u;
        leafmask |= (hit && !inner) ? (1u << i) : 0u;
        const bool ih = hit && inner;
        const uint32_t c = v.child_base + __popc(v.imask & ((1u << i) - 1u));
        const bool first = ih && next == PT_NO_HIT;
        if (ih && !first) stack[st.sp++] = c;
        next = first ? c : next;
    }
    if (st.sp > PT_STACK) { atomicOr(S.err, 1u); st.hit = true; return true; }
    while (leafmask) {
        const int i = __ffs(leafmask) - 1;
        leafmask &= leafmask - 1u;
        const uint32_t meta = byte_of(v.meta_lo, v.meta_hi, i);
        const uint32_t first = v.tri_base + (meta & 31u);
        const uint32_t cnt = meta >> 5;
        for (uint32_t k = 0; k < cnt; ++k) {
            const uint32_t ti = first + k;
            if (COUNT) tc.tris++;
            const float4 a = __ldg(S.tris + 3u * ti), b = __ldg(S.tris + 3u * ti + 1), c = __ldg(S.tris + 3u * ti + 2);
            float t, u, w;
            if (tri_hit(st.wr, xyz(a), xyz(b), xyz(c), st.tmax, t, u, w)) { st.hit = true; return true; }
        }
    }
    if (next != PT_NO_HIT) {
        st.node = next;
        return false;
    }
    if (st.sp == 0) return true;
    st.node = stack[--st.sp];
    return false;
}

template <bool COUNT>
__device__ __forceinline__ bool trace_any_t(const DScene& S, float3 o, float3 d, float tmax, TravCount& tc) {
    AnyState st;
    uint32_t stack[PT_STACK + PT_STACK_SLACK];
    any_init(S, o, d, tmax, st);
    while (!any_step<COUNT>(S, st, stack, tc)) {
    }
    return st.hit;
}

// ---- cooperative traversal: one ray per group of 8 lanes ----
// The per-lane traversal above keeps a warp's 32 rays in 32 lanes; rays need different numbers
// of nodes and leaves, so most lanes idle (about 9 of 32 active per instruction on the 1080p
// CAD frame).  Here a group of COOP_W = 8 lanes carries one ray (4 rays per warp): lane j of
// the group tests child slot j of the node, and the triangles of the node's hit leaves are
// spread over the group's lanes.  The group visits exactly the nodes the per-lane traversal
// visits, in the same order: the same box tests against the same current closest t, the same
// nearest child descended into, and the other hit children pushed in the same order -- the
// per-lane loop pushes, at each later internal hit, either that child or (when it is nearer
// than every earlier one) the previous nearest; an exclusive prefix minimum over the group's
// lanes gives each lane what the loop pushes at its slot and where.  So the hit, and the node
// and triangle counts of the counting variant, equal the per-lane traversal's.
constexpr uint32_t COOP_W = 8;
constexpr uint32_t COOP_LIST = 64;   // triangle slots: 8 leaves of at most 7 triangles

// per group, in shared memory: the node stack (node, entry t bits) and the hit leaves'
// triangle list of the current node
struct CoopShared {
    uint2 stack[PT_STACK];
    uint32_t list[COOP_LIST];
};

struct CoopClosest {
    WRay wr;
    TravRay tr;
    float tmax;
    float hit_t;                      // the group's closest t so far (the same in every lane)
    uint32_t node, budget;
    int sp;
    bool fail;
    float bt, bu, bv;                 // this lane's closest hit among the triangles it tested
    uint32_t btri, borig;
};

__device__ __forceinline__ void coop_closest_init(const DScene& S, float3 o, float3 d, float tmax, CoopClosest& st) {
    st.wr = make_wray(o, d);
    st.tr = make_trav(o, d);
    st.tmax = tmax;
    st.hit_t = tmax;
    st.node = 0;
    st.sp = 0;
    st.fail = false;
    st.budget = (uint32_t)S.n_nodes + 1u;
    st.bt = tmax;
    st.bu = st.bv = 0.0f;
    st.btri = PT_NO_HIT;
    st.borig = PT_NO_HIT;
}

// box test of this lane's child slot; ib / lb: the group's internal / leaf hits (slot bits)
__device__ __forceinline__ float coop_node_test(const NodeView& v, const TravRay& tr, float tmax, uint32_t gl,
                                                uint32_t gm, uint32_t gbase, uint32_t& meta, uint32_t& ib,
                                                uint32_t& lb) {
    meta = byte_of(v.meta_lo, v.meta_hi, (int)gl);
    float tn = -1.0f;
    if (meta != 0u) {
        NodeTest T;
        node_setup(v, tr, T);
        tn = child_test(T, (int)gl, tmax);
    }
    const bool hit = meta != 0u && tn >= 0.0f && tn <= tmax;
    const bool is_int = (v.imask >> gl) & 1u;
    ib = (__ballot_sync(gm, hit && is_int) >> gbase) & 0xffu;
    lb = (__ballot_sync(gm, hit && !is_int) >> gbase) & 0xffu;
    return tn;
}

// the triangles of the hit leaves (slot order, then triangle order) into the group's list;
// returns their number
__device__ __forceinline__ uint32_t coop_leaf_list(const NodeView& v, uint32_t meta, uint32_t lb, uint32_t gl,
                                                   uint32_t gm, uint32_t* list) {
    const uint32_t cnt = ((lb >> gl) & 1u) ? (meta >> 5) : 0u;
    uint32_t x = cnt;
#pragma unroll
    for (uint32_t d = 1; d < COOP_W; d <<= 1) {
        const uint32_t y = __shfl_up_sync(gm, x, d, COOP_W);
        if (gl >= d) x += y;
    }
    const uint32_t total = __shfl_sync(gm, x, COOP_W - 1, COOP_W);
    const uint32_t first = v.tri_base + (meta & 31u);
    for (uint32_t k = 0; k < cnt; ++k) list[x - cnt + k] = first + k;
    __syncwarp(gm);
    return total;
}

// one node of the closest-hit traversal by the group; true once the ray is finished
template <bool COUNT>
__device__ __forceinline__ bool coop_closest_step(const DScene& S, CoopClosest& st, CoopShared& sh, uint32_t gl,
                                                  uint32_t gm, uint32_t gbase, TravCount& tc) {
    __syncwarp(gm);   // the last pop's read of the stack comes before this node's pushes
    if (S.n_nodes == 0) return true;
    if (st.budget-- == 0u) {
        if (gl == 0) atomicOr(S.err, 4u);
        st.fail = true;
        return true;
    }
    const NodeView v = load_node(S.nodes, st.node);
    if (COUNT && gl == 0) { tc.nodes++; tc.boxes += node_slots(v); }
    uint32_t meta, ib, lb;
    const float tn = coop_node_test(v, st.tr, st.hit_t, gl, gm, gbase, meta, ib, lb);
    const bool ih = (ib >> gl) & 1u;
    const uint32_t child = v.child_base + __popc(v.imask & ((1u << gl) - 1u));
    // inclusive prefix minimum of (t, child) over the internal hits in slot order; a later
    // hit displaces an earlier one only when strictly nearer
    float pt = ih ? tn : __int_as_float(0x7f800000);
    uint32_t pc = child;
#pragma unroll
    for (uint32_t d = 1; d < COOP_W; d <<= 1) {
        const float t2 = __shfl_up_sync(gm, pt, d, COOP_W);
        const uint32_t c2 = __shfl_up_sync(gm, pc, d, COOP_W);
        if (gl >= d && !(pt < t2)) { pt = t2; pc = c2; }
    }
    float ex_t = __shfl_up_sync(gm, pt, 1, COOP_W);
    const uint32_t ex_c = __shfl_up_sync(gm, pc, 1, COOP_W);
    if (gl == 0) ex_t = __int_as_float(0x7f800000);
    const float near_t = __shfl_sync(gm, pt, COOP_W - 1, COOP_W);
    const uint32_t near_c = __shfl_sync(gm, pc, COOP_W - 1, COOP_W);
    // the j-th internal hit (j >= 1) pushes the displaced nearest or itself at stack slot sp + j - 1
    const uint32_t n_int = __popc(ib);
    const uint32_t n_push = n_int > 0u ? n_int - 1u : 0u;
    if (st.sp + (int)n_push > PT_STACK) {
        if (gl == 0) atomicOr(S.err, 1u);
        st.fail = true;
        return true;
    }
    const uint32_t j = __popc(ib & ((1u << gl) - 1u));
    if (ih && j > 0u) {
        const bool displaces = tn < ex_t;
        sh.stack[st.sp + (int)j - 1] = displaces ? make_uint2(ex_c, __float_as_uint(ex_t))
                                                 : make_uint2(child, __float_as_uint(tn));
    }
    st.sp += (int)n_push;
    if (lb) {
        const uint32_t total = coop_leaf_list(v, meta, lb, gl, gm, sh.list);
        if (COUNT && gl == 0) tc.tris += total;
        for (uint32_t b = 0; b < total; b += COOP_W) {
            const uint32_t q = b + gl;
            if (q < total) {
                const uint32_t ti = sh.list[q];
                const float4 a = __ldg(S.tris + 3u * ti), bb = __ldg(S.tris + 3u * ti + 1), c = __ldg(S.tris + 3u * ti + 2);
                float t, u, w;
                if (tri_hit(st.wr, xyz(a), xyz(bb), xyz(c), st.tmax, t, u, w)) {
                    const uint32_t orig = __float_as_uint(a.w);
                    if (t < st.bt || (t == st.bt && orig < st.borig)) {
                        st.bt = t; st.bu = u; st.bv = w; st.btri = ti; st.borig = orig;
                    }
                }
            }
        }
        // t > 0 and +inf order like their bit patterns
        st.hit_t = __uint_as_float(__reduce_min_sync(gm, __float_as_uint(st.bt)));
    }
    __syncwarp(gm);   // the pushes and the list are read by other lanes of the group
    if (n_int > 0u && near_t <= st.hit_t) {
        st.node = near_c;
        return false;
    }
    while (st.sp > 0) {
        const uint2 e = sh.stack[--st.sp];
        if (__uint_as_float(e.y) <= st.hit_t) { st.node = e.x; return false; }
    }
    return true;
}

// the group's hit: the lexicographic minimum of (t, original triangle id) over its lanes.
// Returns true in the one lane that holds it (lane 0 of the group for a miss).
__device__ __forceinline__ bool coop_closest_finish(const CoopClosest& st, uint32_t gl, uint32_t gm, uint32_t gbase,
                                                    HitRec& h) {
    const uint32_t tb = __reduce_min_sync(gm, __float_as_uint(st.bt));
    const bool at_t = __float_as_uint(st.bt) == tb && st.btri != PT_NO_HIT;
    const uint32_t ob = __reduce_min_sync(gm, at_t ? st.borig : 0xffffffffu);
    const uint32_t wl = (__ballot_sync(gm, at_t && st.borig == ob) >> gbase) & 0xffu;
    const bool fail = st.fail;
    if (wl == 0u || fail) {
        h.t = fail ? st.hit_t : st.tmax;
        h.u = h.v = 0.0f;
        h.tri = PT_NO_HIT;
        return gl == 0u;
    }
    h.t = st.bt; h.u = st.bu; h.v = st.bv; h.tri = st.btri;
    return gl == (uint32_t)(__ffs(wl) - 1);
}

struct CoopAny {
    WRay wr;
    TravRay tr;
    float tmax;
    uint32_t node, budget;
    int sp;
    bool hit;
};

__device__ __forceinline__ void coop_any_init(const DScene& S, float3 o, float3 d, float tmax, CoopAny& st) {
    st.wr = make_wray(o, d);
    st.tr = make_trav(o, d);
    st.tmax = tmax;
    st.node = 0;
    st.sp = 0;
    st.hit = false;
    st.budget = (uint32_t)S.n_nodes + 1u;
}

// one node of the any-hit traversal by the group (the per-lane order: the first internal hit
// in slot order next, the others pushed in slot order; leaf triangles in slot order, counted
// up to the first hit); true once the ray is finished (st.hit: occluded)
template <bool COUNT>
__device__ __forceinline__ bool coop_any_step(const DScene& S, CoopAny& st, CoopShared& sh, uint32_t gl, uint32_t gm,
                                              uint32_t gbase, TravCount& tc) {
    __syncwarp(gm);   // the last pop's read of the stack comes before this node's pushes
    if (S.n_nodes == 0) return true;
    if (st.budget-- == 0u) {
        if (gl == 0) atomicOr(S.err, 4u);
        return true;
    }
    const NodeView v = load_node(S.nodes, st.node);
    if (COUNT && gl == 0) { tc.nodes++; tc.boxes += node_slots(v); }
    uint32_t meta, ib, lb;
    coop_node_test(v, st.tr, st.tmax, gl, gm, gbase, meta, ib, lb);
    const uint32_t n_int = __popc(ib);
    const uint32_t n_push = n_int > 0u ? n_int - 1u : 0u;
    if (st.sp + (int)n_push > PT_STACK) {
        if (gl == 0) atomicOr(S.err, 1u);
        st.hit = true;
        return true;
    }
    const uint32_t child = v.child_base + __popc(v.imask & ((1u << gl) - 1u));
    const uint32_t j = __popc(ib & ((1u << gl) - 1u));
    if (((ib >> gl) & 1u) && j > 0u) sh.stack[st.sp + (int)j - 1].x = child;
    const uint32_t first_slot = ib ? (uint32_t)(__ffs(ib) - 1) : 0u;
    const uint32_t next = __shfl_sync(gm, child, first_slot, COOP_W);
    st.sp += (int)n_push;
    if (lb) {
        const uint32_t total = coop_leaf_list(v, meta, lb, gl, gm, sh.list);
        for (uint32_t b = 0; b < total; b += COOP_W) {
            const uint32_t q = b + gl;
            bool h = false;
            if (q < total) {
                const uint32_t ti = sh.list[q];
                const float4 a = __ldg(S.tris + 3u * ti), bb = __ldg(S.tris + 3u * ti + 1), c = __ldg(S.tris + 3u * ti + 2);
                float t, u, w;
                h = tri_hit(st.wr, xyz(a), xyz(bb), xyz(c), st.tmax, t, u, w);
            }
            const uint32_t hm = (__ballot_sync(gm, h) >> gbase) & 0xffu;
            if (hm) {
                if (COUNT && gl == 0) tc.tris += b + (uint32_t)__ffs(hm);
                st.hit = true;
                return true;
            }
        }
        if (COUNT && gl == 0) tc.tris += total;
    }
    __syncwarp(gm);
    if (n_int > 0u) {
        st.node = next;
        return false;
    }
    if (st.sp == 0) return true;
    st.node = sh.stack[--st.sp].x;
    return false;
}

// out-of-line entry points keep the megakernel's code and registers in check
static __device__ __noinline__ void trace_closest(const DScene& S, float3 o, float3 d, float tmax, HitRec& h) {
    TravCount tc;
    trace_closest_t<false, true>(S, o, d, tmax, h, tc);
}
static __device__ __noinline__ bool trace_any(const DScene& S, float3 o, float3 d, float tmax) {
    TravCount tc;
    return trace_any_t<false>(S, o, d, tmax, tc);
}

// ------------------------------------------------------------------ environment
__device__ __forceinline__ void env_texel(const DScene& S, float3 d, int& x, int& y) {
    const float u = 0.5f + atan2f(d.x, -d.z) * (0.5f * PT_INV_PI_F);
    const float dy = fminf(fmaxf(d.y, -1.0f), 1.0f);
    const float v = acosf(dy) * PT_INV_PI_F;
    int ix = (int)floorf(u * (float)S.env_w), iy = (int)floorf(v * (float)S.env_h);
    ix = min(max(ix, 0), S.env_w - 1);
    iy = min(max(iy, 0), S.env_h - 1);
    x = ix;
    y = iy;
}
__device__ __forceinline__ float3 env_radiance(const DScene& S, float3 d) {
    int x, y;
    env_texel(S, d, x, y);
    const float* t = S.env + 3 * ((size_t)y * S.env_w + x);
    return mk3(t[0], t[1], t[2]);
}
__device__ __forceinline__ float env_pdf(const DScene& S, float3 d) {
    if (S.env_total <= 0.0f) return 0.0f;
    int x, y;
    env_texel(S, d, x, y);
    const float s = sqrtf(fmaxf(0.0f, 1.0f - d.y * d.y));
    if (s <= 0.0f) return 0.0f;
    const float pdf_uv = S.env_wtex[(size_t)y * S.env_w + x] / S.env_total * (float)S.env_w * (float)S.env_h;
    return pdf_uv / (2.0f * PT_PI_F * PT_PI_F * s);
}
// largest i in [0, n-1] with cdf[i] <= u
// the largest i in [lo, hi] with cdf[i] <= u, given cdf[lo] <= u (cdf non-decreasing)
__device__ __forceinline__ int cdf_find_in(const float* cdf, int lo, int hi, float u) {
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(cdf + mid) <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ int cdf_find(const float* cdf, int n, float u) { return cdf_find_in(cdf, 0, n - 1, u); }

// The same index through a guide table (the cutpoint method of Chen and Asau 1974): guide[g] is
// the answer for u = g / G, G a power of two, so g = floor(u G) is exact and the answer for u
// lies in [guide[g], guide[g + 1]]: the search there returns what the search over [0, n - 1]
// returns, in about one step instead of log2 n dependent loads.
__device__ __forceinline__ int cdf_find_guided(const float* cdf, const int* guide, int G, float u) {
    const int g = min(max((int)(u * (float)G), 0), G - 1);
    return cdf_find_in(cdf, __ldg(guide + g), __ldg(guide + g + 1), u);
}
__device__ __forceinline__ bool env_sample(const DScene& S, float u3, float u4, float3& d, float& pdf, float3& L) {
    if (S.env_total <= 0.0f) return false;
    const int w = S.env_w, h = S.env_h;
    const int y = cdf_find_guided(S.env_marg, S.env_guide, S.env_gm, u3);
    const float m0 = S.env_marg[y], m1 = S.env_marg[y + 1];
    const float dv = m1 > m0 ? (u3 - m0) / (m1 - m0) : 0.5f;
    const float* cd = S.env_cond + (size_t)y * (w + 1);
    const int x = cdf_find_guided(cd, S.env_guide + (S.env_gm + 1) + (size_t)y * (S.env_gc + 1), S.env_gc, u4);
    const float c0 = cd[x], c1 = cd[x + 1];
    const float du = c1 > c0 ? (u4 - c0) / (c1 - c0) : 0.5f;
    const float u = ((float)x + du) / (float)w, v = ((float)y + dv) / (float)h;
    const float theta = v * PT_PI_F, phi = (u - 0.5f) * 2.0f * PT_PI_F;
    float st, ct, sp, cp;
    sincosf(theta, &st, &ct);
    sincosf(phi, &sp, &cp);
    if (st <= 0.0f) return false;
    d = mk3(st * sp, ct, -st * cp);
    const float pdf_uv = S.env_wtex[(size_t)y * w + x] / S.env_total * (float)w * (float)h;
    pdf = pdf_uv / (2.0f * PT_PI_F * PT_PI_F * st);
    const float* t = S.env + 3 * ((size_t)y * w + x);
    L = mk3(t[0], t[1], t[2]);
    return pdf > 0.0f;
}

// ------------------------------------------------------------------ camera
struct DCam {
    float3 origin, target, up;
    float vfov_deg;
    uint32_t width, height;
    float lens_radius, focus_distance;   // thin lens; radius 0 = pinhole
};

// Concentric map of the unit square onto the unit disk (Shirley and Chiu 1997): square rings
// go to disk rings, so uniform points stay uniform.
__device__ __forceinline__ void concentric_disk(float u0, float u1, float& x, float& y) {
    const float a = 2.0f * u0 - 1.0f, b = 2.0f * u1 - 1.0f;
    if (a == 0.0f && b == 0.0f) { x = 0.0f; y = 0.0f; return; }
    float r, phi;
    if (fabsf(a) > fabsf(b)) { r = a; phi = (0.25f * PT_PI_F) * (b / a); }
    else { r = b; phi = 0.5f * PT_PI_F - (0.25f * PT_PI_F) * (a / b); }
    x = r * cosf(phi);
    y = r * sinf(phi);
}

// Camera ray of pixel (px, py) with jitter (u0, u1) and lens uniforms (l0, l1), the latter
// used only by a thin lens: the ray starts at the lens point and passes through the point
// where the pinhole ray of the same jitter meets the plane of focus.
__device__ __forceinline__ void camera_ray(const DCam& c, uint32_t px, uint32_t py, float u0, float u1, float l0,
                                           float l1, float3& o, float3& d) {
    const float3 fwd = norm3(c.target - c.origin);
    const float3 right = norm3(cross3(fwd, c.up));
    const float3 up = cross3(right, fwd);
    const float th = tanf(0.5f * c.vfov_deg * (PT_PI_F / 180.0f));
    const float aspect = (float)c.width / (float)c.height;
    const float nx = (2.0f * ((float)px + u0) / (float)c.width - 1.0f) * aspect * th;
    const float ny = (1.0f - 2.0f * ((float)py + u1) / (float)c.height) * th;
    const float3 dp = norm3(fwd + right * nx + up * ny);
    if (c.lens_radius > 0.0f) {
        float lx, ly;
        concentric_disk(l0, l1, lx, ly);
        const float3 focus = c.origin + dp * (c.focus_distance / dot3(dp, fwd));
        const float3 lens = c.origin + (right * (c.lens_radius * lx) + up * (c.lens_radius * ly));
        o = lens;
        d = norm3(focus - lens);
        return;
    }
    o = c.origin;
    d = dp;
}

// the camera ray of pixel (px, py) = pixel id p, sample s: jitter from dimensions 0-1 and,
// for a thin lens, the lens point from dimensions 12-13 of the first vertex
constexpr uint32_t DIM_LENS = 12;
__device__ __forceinline__ void camera_ray_ps(const DCam& c, uint32_t px, uint32_t py, uint32_t p, uint32_t s,
                                              uint32_t k0, uint32_t k1, float3& o, float3& d) {
    const uint4 u = philox4x32_10(make_uint4(p, s, 0u, 0u), k0, k1);
    float l0 = 0.0f, l1 = 0.0f;
    if (c.lens_radius > 0.0f) {
        const uint4 w = philox4x32_10(make_uint4(p, s, 0u, DIM_LENS >> 2), k0, k1);
        l0 = u24(w.x);
        l1 = u24(w.y);
    }
    camera_ray(c, px, py, u24(u.x), u24(u.y), l0, l1, o, d);
}

__device__ __forceinline__ float3 offset_origin(float3 x, float3 ng, float3 dir, float eps) {
    const float s = dot3(dir, ng) > 0.0f ? 1.0f : -1.0f;
    return x + ng * (s * eps);
}

// ------------------------------------------------------------------ one path vertex
// Path state carried between bounces.
struct PathState {
    float3 beta;
    float3 L;
    float prev_pdf;     // mixture pdf of the last BSDF sample; < 0 after a delta lobe / camera
};

struct ShadowRay {
    float3 o, d, contrib;
    float tmax;
};

enum { FLAG_NO_NEE = 1u, FLAG_NO_RR = 2u, FLAG_COUNT = 4u, FLAG_RESTIR = 1u << 16 /* internal */ };

// ------------------------------------------------------------------ ReSTIR DI (primary vertex)
// Reservoir resampling of light samples (Bitterli et al. 2020), which the paper names as
// future work for many lights (Sec. 2, Sec. 6.3).  A light sample is (light, y): a quad
// index and a point on it (area measure), or LIGHT_ENV and a direction (solid angle).
// Reservoir records: float4 (y, light bits), float4 (W, M, target at the owner, 0).
constexpr uint32_t RESTIR_CANDIDATES = 0xFFFF0001u, RESTIR_SPATIAL = 0xFFFF0002u;
constexpr int LIGHT_NONE = -2, LIGHT_ENV = -1;

// Unshadowed contribution c = f(wo, w_y) L_e(y) |cos| G(y) of light sample (light, y) at the
// surface point x with frame (tt, bb, n) and closure C (G = cos_l / d^2 on a quad, 1 for the
// environment); returns the target, the luminance of c (0 where the light cannot reach x).
__device__ __forceinline__ float restir_target(const DScene& S, float3 x, float3 tt, float3 bb, float3 n,
                                               const Closure& C, float3 wo, int light, float3 y, float3& c,
                                               float3& ld) {
    float3 Le;
    float geo;
    c = splat3(0.0f);
    ld = splat3(0.0f);
    if (light >= 0) {
        const DQuad& q = S.quads[light];
        const float3 to = y - x;
        const float d2 = dot3(to, to);
        if (!(d2 > 0.0f)) return 0.0f;
        ld = to * (1.0f / sqrtf(d2));
        const float cl = -dot3(ld, q.n);
        if (!(cl > 0.0f || (q.two_sided && cl < 0.0f))) return 0.0f;
        Le = q.L;
        geo = fabsf(cl) / d2;
    } else if (light == LIGHT_ENV) {
        ld = y;
        Le = env_radiance(S, ld);
        geo = 1.0f;
    } else {
        return 0.0f;
    }
    const float3 wl = mk3(dot3(ld, tt), dot3(ld, bb), dot3(ld, n));
    float3 f;
    float pdf;
    closure_eval(C, wo, wl, f, pdf);
    c = (f * Le) * (fabsf(wl.z) * geo);
    const float ph = lum3(c);
    return (ph > 0.0f && isfinite(ph)) ? ph : 0.0f;
}

// Cheap target p0 of the initial candidates: lum(L_e) G |cos| on the side the surface
// scatters to (above it; both sides if it transmits).  Its support holds that of the
// contribution, so resampling with it keeps the reservoir unbiased (generalised RIS).
__device__ __forceinline__ float restir_target0(const DScene& S, float3 x, float3 n, bool transmits, int light,
                                                float3 y) {
    float3 ld, Le;
    float geo;
    if (light >= 0) {
        const DQuad& q = S.quads[light];
        const float3 to = y - x;
        const float d2 = dot3(to, to);
        if (!(d2 > 0.0f)) return 0.0f;
        ld = to * (1.0f / sqrtf(d2));
        const float cl = -dot3(ld, q.n);
        if (!(cl > 0.0f || (q.two_sided && cl < 0.0f))) return 0.0f;
        Le = q.L;
        geo = fabsf(cl) / d2;
    } else if (light == LIGHT_ENV) {
        ld = y;
        Le = env_radiance(S, ld);
        geo = 1.0f;
    } else {
        return 0.0f;
    }
    const float c = dot3(ld, n);
    if (!(c > 0.0f) && !(transmits && c < 0.0f)) return 0.0f;
    const float ph = lum3(Le) * geo * fabsf(c);
    return (ph > 0.0f && isfinite(ph)) ? ph : 0.0f;
}

constexpr uint32_t RESTIR_LATER = 0xFFFF0100u;   // + vertex index: candidates at vertex k >= 1

// Resampled importance sampling of M light candidates from the next-event light sampler
// (candidate i: Philox block (p, s, stream, i) = light pick, u, v, selection) with the cheap
// target p0; the kept sample (light, y) has the unbiased contribution weight
// W = sum w / (M p0(y)), w = p0 / source pdf (area measure on a quad, solid angle for the sky).
__device__ __forceinline__ void restir_ris(const DScene& S, float3 x, float3 n, bool transmits, uint32_t p, uint32_t s,
                                           uint32_t stream, uint32_t M, uint32_t k0, uint32_t k1, int& sel,
                                           float3& y_sel, float& W, float& ph_sel) {
    const bool has_env = S.env_w > 0 && S.env_total > 0.0f;
    const float p_env = has_env ? (S.n_quads > 0 ? 0.5f : 1.0f) : 0.0f;
    float wsum = 0.0f;
    sel = LIGHT_NONE;
    y_sel = splat3(0.0f);
    ph_sel = 0.0f;
    for (uint32_t i = 0; i < M; ++i) {
        const uint4 r = philox4x32_10(make_uint4(p, s, stream, i), k0, k1);
        const float u_pick = u24(r.x), u = u24(r.y), v = u24(r.z), u_sel = u24(r.w);
        int light;
        float3 y;
        float src;
        if (u_pick < p_env) {
            float pe;
            float3 Ld;
            if (!env_sample(S, u, v, y, pe, Ld)) continue;
            light = LIGHT_ENV;
            src = p_env * pe;
        } else {
            int l = (int)floorf((u_pick - p_env) / (1.0f - p_env) * (float)S.n_quads);
            l = min(l, S.n_quads - 1);
            const DQuad& q = S.quads[l];
            light = l;
            y = q.p0 + q.e1 * u + q.e2 * v;
            src = (1.0f - p_env) / (float)S.n_quads / q.area;
        }
        if (!(src > 0.0f)) continue;
        const float ph = restir_target0(S, x, n, transmits, light, y);
        const float w = ph / src;
        if (!(w > 0.0f)) continue;
        wsum += w;
        if (u_sel * wsum < w) {
            sel = light;
            y_sel = y;
            ph_sel = ph;
        }
    }
    W = (sel != LIGHT_NONE && ph_sel > 0.0f) ? wsum / ((float)M * ph_sel) : 0.0f;
}

// The primary surface of a path as the reservoirs see it, rebuilt from its position, the
// direction towards the camera and the triangle (the same steps as shade_vertex_h).
struct RSurf {
    float3 x, n, tt, bb, wo;
    Closure C;
};
__device__ __forceinline__ void rsurf_make(const DScene& S, float3 x, float3 wo_w, uint32_t tri, RSurf& g) {
    const float4 ta = __ldg(S.tris + 3u * tri), tb = __ldg(S.tris + 3u * tri + 1), tc = __ldg(S.tris + 3u * tri + 2);
    const float3 ng = norm3(cross3(xyz(tb) - xyz(ta), xyz(tc) - xyz(ta)));
    const bool front = dot3(wo_w, ng) > 0.0f;
    const uint32_t mid = __float_as_uint(tb.w);
    const DMat M = S.mats[mid];
    g.x = x;
    g.n = front ? ng : -ng;
    if (M.spec_aniso > 0.0f) tangent_frame(g.n, xyz(tb) - xyz(ta), M.spec_rot, g.tt, g.bb);
    else onb(g.n, g.tt, g.bb);
    g.wo = mk3(dot3(wo_w, g.tt), dot3(wo_w, g.bb), dot3(wo_w, g.n));
    closure_setup(g.C, M, front, g.wo.z, S.fuzz + FUZZ_FLOATS * mid);
}

enum ShadeResult { SHADE_END = 0, SHADE_CONTINUE = 1 };

struct ShadeOut {
    float3 next_o, next_d;
    bool has_shadow;
    ShadowRay sh;
    bool rr_end;
};

// Vertex hook of the plain tracer: never ends a path.
struct NoHook {
    __device__ __forceinline__ bool operator()(float3, float3, float3, const DMat&, const PathState&, uint32_t) {
        return false;
    }
};

// Handles the hit (or miss) of the ray (o, d) at path vertex k: emission with MIS, the
// depth limit, next-event estimation (returned as a shadow ray whose contribution is
// added if unoccluded), BSDF sampling and Russian roulette.  Returns SHADE_CONTINUE with
// the next ray, or SHADE_END.  `hook` sees every scattering vertex below the depth limit
// (position, direction to the previous vertex, shading normal, material, path state) and
// may end the path there (the radiance cache does).
// RIS: the ReSTIR DI branches (vertex 0 from its reservoir, later vertices by resampled
// candidates, zero-weighted light hits) are compiled in only where a ReSTIR render runs.
template <class Hook, bool RIS = false, bool FUZZ = true>
__device__ __forceinline__ int shade_vertex_h(const DScene& S, const HitRec& h, float3 o, float3 d, uint32_t k,
                                              uint32_t max_depth, uint32_t flags, const VertexRng& rng,
                                              PathState& ps, ShadeOut& out, Hook& hook,
                                              const float4* rres = nullptr, uint32_t later_m = 0) {
    out.has_shadow = false;
    out.rr_end = false;
    const bool nee = !(flags & FLAG_NO_NEE);
    const bool has_env = S.env_w > 0 && S.env_total > 0.0f;
    const float p_env = has_env ? (S.n_quads > 0 ? 0.5f : 1.0f) : 0.0f;
    const bool prev_delta = ps.prev_pdf < 0.0f;
    // with ReSTIR DI the reservoir at vertex 0 (and, with later candidates, the resampled
    // estimate at every later vertex) estimates all light arriving there: a light reached by
    // BSDF sampling from such a vertex counts with weight 0 (1 after a delta lobe)
    const bool restir1 = RIS && (flags & FLAG_RESTIR) && (k == 1 || (k > 1 && later_m > 0));
    if (h.tri == PT_NO_HIT) {
        if (has_env) {
            const float3 Le = env_radiance(S, d);
            float w = 1.0f;
            if (!prev_delta && nee) w = restir1 ? 0.0f : power_heuristic(ps.prev_pdf, p_env * env_pdf(S, d));
            ps.L = ps.L + (ps.beta * Le) * w;
        }
        return SHADE_END;
    }
    const float4 ta = __ldg(S.tris + 3u * h.tri), tb = __ldg(S.tris + 3u * h.tri + 1), tc = __ldg(S.tris + 3u * h.tri + 2);
    const float3 x = o + d * h.t;
    const float3 ng = norm3(cross3(xyz(tb) - xyz(ta), xyz(tc) - xyz(ta)));
    const float3 wo_w = -d;
    const bool front = dot3(wo_w, ng) > 0.0f;
    const uint32_t code = __float_as_uint(tb.w);
    if (code & PT_LIGHT_BIT) {
        const DQuad& q = S.quads[code & ~PT_LIGHT_BIT];
        const float cl = dot3(wo_w, q.n);
        if (cl > 0.0f || (q.two_sided && cl < 0.0f)) {
            float w = 1.0f;
            if (!prev_delta && nee) {
                const float pl = (1.0f - p_env) / (float)S.n_quads * h.t * h.t / (q.area * fabsf(cl));
                w = restir1 ? 0.0f : power_heuristic(ps.prev_pdf, pl);
            }
            ps.L = ps.L + (ps.beta * q.L) * w;
        }
        return SHADE_END;
    }
    const DMat M = S.mats[code];
    if (front && (M.emission.x > 0.0f || M.emission.y > 0.0f || M.emission.z > 0.0f))
        ps.L = ps.L + ps.beta * M.emission;
    if (k == max_depth) return SHADE_END;

    const float3 n = front ? ng : -ng;
    float3 tt, bb;
    if (M.spec_aniso > 0.0f) tangent_frame(n, xyz(tb) - xyz(ta), M.spec_rot, tt, bb);
    else onb(n, tt, bb);
    const float3 wo = mk3(dot3(wo_w, tt), dot3(wo_w, bb), dot3(wo_w, n));
    if (hook(x, wo_w, n, M, ps, k)) return SHADE_END;
    Closure C;
    closure_setup<FUZZ>(C, M, front, wo.z, S.fuzz + FUZZ_FLOATS * code);

    const uint4 r0 = rng.block(0), r1 = rng.block(1), r2 = rng.block(2);
    if (RIS && (flags & FLAG_RESTIR) && k == 0) {
        // the sample of the path's final reservoir in place of next-event estimation
        if (rres != nullptr) {
            const float4 ry = rres[0], rw = rres[1];
            const int light = __float_as_int(ry.w);
            if (light != LIGHT_NONE && rw.x > 0.0f) {
                float3 c, ld;
                if (restir_target(S, x, tt, bb, n, C, wo, light, xyz(ry), c, ld) > 0.0f) {
                    const float3 so = offset_origin(x, ng, ld, S.eps);
                    float3 sd = ld;
                    float tmax = __int_as_float(0x7f800000);
                    if (light >= 0) {
                        const float3 to = xyz(ry) - so;
                        const float dl = len3(to);
                        sd = to * (1.0f / dl);
                        tmax = (1.0f - 1e-4f) * dl;
                    }
                    out.has_shadow = true;
                    out.sh.o = so;
                    out.sh.d = sd;
                    out.sh.tmax = tmax;
                    out.sh.contrib = (ps.beta * c) * rw.x;
                }
            }
        }
    } else if (RIS && (flags & FLAG_RESTIR) && later_m > 0 && C.has_smooth && (has_env || S.n_quads > 0)) {
        // resampled light candidates at a later vertex (no reuse)
        int light;
        float3 yk;
        float Wk, ph0;
        restir_ris(S, x, n, (1.0f - C.m) * C.t > 0.0f, rng.p, rng.s, RESTIR_LATER + k, later_m, rng.k0, rng.k1, light,
                   yk, Wk, ph0);
        if (light != LIGHT_NONE && Wk > 0.0f) {
            float3 c, ld;
            if (restir_target(S, x, tt, bb, n, C, wo, light, yk, c, ld) > 0.0f) {
                const float3 so = offset_origin(x, ng, ld, S.eps);
                float3 sd = ld;
                float tmax = __int_as_float(0x7f800000);
                if (light >= 0) {
                    const float3 to = yk - so;
                    const float dl = len3(to);
                    sd = to * (1.0f / dl);
                    tmax = (1.0f - 1e-4f) * dl;
                }
                out.has_shadow = true;
                out.sh.o = so;
                out.sh.d = sd;
                out.sh.tmax = tmax;
                out.sh.contrib = (ps.beta * c) * Wk;
            }
        }
    } else if (nee && C.has_smooth && (has_env || S.n_quads > 0)) {
        const float u2 = u24(r0.z), u3 = u24(r0.w), u4 = u24(r1.x);
        float3 ld, Le = splat3(0.0f), ly = splat3(0.0f);
        float pl = 0.0f;
        bool ok = false, to_quad = false;
        if (u2 < p_env) {
            float pe;
            if (env_sample(S, u3, u4, ld, pe, Le)) {
                pl = p_env * pe;
                ok = true;
            }
        } else {
            int l = (int)floorf((u2 - p_env) / (1.0f - p_env) * (float)S.n_quads);
            l = min(l, S.n_quads - 1);
            const DQuad& q = S.quads[l];
            const float3 y = q.p0 + q.e1 * u3 + q.e2 * u4;
            const float3 to = y - x;
            const float dist2 = dot3(to, to), dist = sqrtf(dist2);
            ld = to * (1.0f / dist);
            const float cl = -dot3(ld, q.n);
            if (cl > 0.0f || (q.two_sided && cl < 0.0f)) {
                pl = (1.0f - p_env) / (float)S.n_quads * dist2 / (q.area * fabsf(cl));
                Le = q.L;
                ly = y;
                to_quad = true;
                ok = true;
            }
        }
        if (ok && pl > 0.0f) {
            const float3 wl = mk3(dot3(ld, tt), dot3(ld, bb), dot3(ld, n));
            float3 f;
            float pb;
            closure_eval(C, wo, wl, f, pb);
            if (max3(f) > 0.0f) {
                const float3 so = offset_origin(x, ng, ld, S.eps);
                float3 sd = ld;
                float tmax = __int_as_float(0x7f800000);
                if (to_quad) {
                    const float3 to = ly - so;
                    const float dl = len3(to);
                    sd = to * (1.0f / dl);
                    tmax = (1.0f - 1e-4f) * dl;
                }
                const float w = power_heuristic(pl, pb);
                out.has_shadow = true;
                out.sh.o = so;
                out.sh.d = sd;
                out.sh.tmax = tmax;
                out.sh.contrib = ((ps.beta * f) * Le) * (fabsf(wl.z) * w / pl);
            }
        }
    }
    BsdfSample bs;
    if (!closure_sample(C, wo, u24(r1.y), u24(r1.z), u24(r1.w), u24(r2.x), bs)) return SHADE_END;
    ps.beta = ps.beta * bs.weight;
    if (k >= 3 && !(flags & FLAG_NO_RR)) {
        const float q = fminf(0.95f, max3(ps.beta));
        if (u24(r2.y) >= q) {
            out.rr_end = true;
            return SHADE_END;
        }
        ps.beta = ps.beta * (1.0f / q);
    }
    const float3 wi_w = tt * bs.wi.x + bb * bs.wi.y + n * bs.wi.z;
    out.next_o = offset_origin(x, ng, wi_w, S.eps);
    out.next_d = norm3(wi_w);
    ps.prev_pdf = bs.delta ? -1.0f : bs.pdf;
    return SHADE_CONTINUE;
}

template <bool RIS = false, bool FUZZ = true>
__device__ __forceinline__ int shade_vertex(const DScene& S, const HitRec& h, float3 o, float3 d, uint32_t k,
                                            uint32_t max_depth, uint32_t flags, const VertexRng& rng,
                                            PathState& ps, ShadeOut& out, const float4* rres = nullptr,
                                            uint32_t later_m = 0) {
    NoHook nh;
    return shade_vertex_h<NoHook, RIS, FUZZ>(S, h, o, d, k, max_depth, flags, rng, ps, out, nh, rres, later_m);
}

// "diffuse-ish" measure of a vertex: diffuse lobes count as roughness 1
__device__ __forceinline__ float effective_roughness(const DMat& M) {
    return M.metalness * M.spec_rough + (1.0f - M.metalness) * ((1.0f - M.trans_weight) + M.trans_weight * M.spec_rough);
}

// ------------------------------------------------------------------ Kahan accumulation
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}
