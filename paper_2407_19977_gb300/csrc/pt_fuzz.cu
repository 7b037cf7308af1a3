// pt_fuzz.cu -- per-material series of the fuzz lobe (OpenPBR's fuzz layer; the paper names
// more OpenPBR features as future work, Sec. 6.3).
//
// The lobe is the Charlie distribution D = (2 + 1/a) sin(theta_m)^(1/a) / (2 pi) (Estevez &
// Kulla 2017) with its exact Smith masking, G1 = mu / A(mu), A(mu) = int <w, m>+ D(m) dm.
// Neither A nor the lobe's directional albedo
//   E(mu_o) = int D(h) mu_i / (4 (A(mu_i) mu_o + A(mu_o) mu_i - mu_i mu_o)) dw_i
// has a closed form.  One CTA per material integrates them and stores Chebyshev series:
//   A: 16 terms in x = 2 mu - 1, from A at the 16 Chebyshev points, each a 1-D integral over
//      theta_m with the azimuth done in closed form, split where the circle of azimuths
//      starts to dip below the horizon of w (theta_m = asin(mu));
//   E: 32 terms in x = 2 mu^(1/4) - 1 (E behaves like mu log mu at grazing: in mu^(1/4) the
//      series converges to about 1e-9), from E at the 32 Chebyshev points, each a 2-D
//      integral: the polar range cut at mu_i = c, 4c, 16c, ... up to 1 with c = max(mu_o, 1e-6)
//      (the integrand turns over at mu_i ~ mu_o and D has a kink at the mirror direction),
//      each piece integrated over the polar angle (smooth through the pole), the azimuth over
//      [0, pi] (the integrand is even) cut at pi - min(pi, 8 (mu_o + mu_hi)) next to the mirror
//      direction; A(mu_i) from its series.
// Everything is FP32.  The rules are Fejer's first rule (nodes cos((2k+1) pi / 2n), weights
// from a cosine sum), whose nodes and weights FP32 evaluates to a few ulp (Newton-iterated
// Gauss-Legendre weights lose up to 1e-3 in FP32 near the ends); sums are Kahan-compensated
// per lane and combined across a warp by TwoSum.  D is evaluated from sin^2 of the
// microfacet angle, formed without cancellation.
#include <cmath>

#include "pt_device.cuh"
#include "pt_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kNA = 48;      // Fejer points per piece of the A integral (theta_m)
constexpr int kNT = 24;      // per polar piece of the E integral
constexpr int kNP = 64;      // per azimuth part of the E integral
constexpr float kFloor = 1e-6f;   // first polar cut of the E integral: max(mu_o, kFloor)

// Kahan-compensated running sum: s - c is the sum of everything added
struct KSum {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// sum over the warp of compensated partial sums: TwoSum of the leading parts, the rounding
// errors and the lanes' compensations carried in a second word
__device__ __forceinline__ float warp_ksum(const KSum& k) {
    float hi = k.s, lo = -k.c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        const float s = hi + h2, bb = s - hi;
        const float e = (hi - (s - bb)) + (h2 - bb);
        hi = s;
        lo = lo + l2 + e;
    }
    return hi + lo;
}

// node k of Fejer's first n-point rule on [-1, 1]: x = cos(theta), theta = (2k+1) pi / (2n),
// w = (2/n) (1 - 2 sum_{j=1}^{n/2} cos(2 j theta) / (4 j^2 - 1)); the cosine arguments are
// reduced in integers (2 j theta = pi m / n, m = j (2k+1) mod 2n) and the sum runs from its
// smallest terms
__device__ void fejer_node(int n, int k, float* x_out, float* w_out) {
    *x_out = cospif((float)(2 * k + 1) / (float)(2 * n));
    KSum s;
    for (int j = n / 2; j >= 1; --j) {
        const int m = (j * (2 * k + 1)) % (2 * n);
        s.add(cospif((float)m / (float)n) / (float)(4 * j * j - 1));
    }
    *w_out = (2.0f / (float)n) * (1.0f - 2.0f * (s.s - s.c));
}

// Charlie D from sin^2 of the microfacet angle
__device__ __forceinline__ float charlie_D_s2(float s2, float alpha) {
    return (2.0f + 1.0f / alpha) * powf(s2, 0.5f / alpha) * (0.5f * PT_INV_PI_F);
}

// Clenshaw sum of n Chebyshev terms (series in shared memory)
__device__ __forceinline__ float cheb_smem(const float* c, int n, float x) {
    float b1 = 0.0f, b2 = 0.0f;
    for (int k = n - 1; k >= 1; --k) {
        const float t = 2.0f * x * b1 - b2 + c[k];
        b2 = b1;
        b1 = t;
    }
    return x * b1 - b2 + c[0];
}

// coefficient k of the n-term Chebyshev interpolant of values v at the points
// cos(pi (j + 1/2) / n): (2/n) sum_j v_j cos(pi k (j + 1/2) / n), halved for k = 0
__device__ float cheb_coef(const float* v, int n, int k) {
    KSum s;
    for (int j = 0; j < n; ++j) {
        const int m = (k * (2 * j + 1)) % (4 * n);
        s.add(v[j] * cospif((float)m / (float)(2 * n)));
    }
    const float c = (2.0f / (float)n) * (s.s - s.c);
    return k == 0 ? 0.5f * c : c;
}

// one material per CTA; raw rows of PT_OPENPBR_FLOATS floats; out FUZZ_FLOATS per row (the
// head fw, fc[3], a, then the A and E series; zeros for a row without fuzz)
__global__ void __launch_bounds__(kThreads) k_fuzz_series(const float* __restrict__ raw, uint32_t n,
                                                          float* __restrict__ out) {
    __shared__ float fa_x[kNA], fa_w[kNA], ft_x[kNT], ft_w[kNT], fp_x[kNP], fp_w[kNP];
    __shared__ float a_val[FUZZ_A_TERMS], e_val[FUZZ_E_TERMS], c_a[FUZZ_A_TERMS];
    __shared__ float piece_mu[kWarps][kNT], piece_s[kWarps][kNT], piece_k[kWarps][kNT];
    const uint32_t row = blockIdx.x;
    if (row >= n) return;
    const float* v = raw + (size_t)PT_OPENPBR_FLOATS * row;
    float* o = out + (size_t)FUZZ_FLOATS * row;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (!(v[29] > 0.0f)) {
        if (t < FUZZ_FLOATS) o[t] = 0.0f;
        return;
    }
    const float r = fmaxf(v[33], 0.2f);
    const float alpha = r * r;
    if (t < FUZZ_HEAD) o[t] = t < 4 ? v[29 + t] : (t == 4 ? alpha : 0.0f);   // fw, fc, a
    if (t < kNA) fejer_node(kNA, t, &fa_x[t], &fa_w[t]);
    else if (t < kNA + kNT) fejer_node(kNT, t - kNA, &ft_x[t - kNA], &ft_w[t - kNA]);
    else if (t < kNA + kNT + kNP) fejer_node(kNP, t - kNA - kNT, &fp_x[t - kNA - kNT], &fp_w[t - kNA - kNT]);
    __syncthreads();

    // A at the Chebyshev points mu_j = (1 + cos(pi (j + 1/2) / 16)) / 2 = cos^2(pi (j + 1/2) / 32):
    // one warp per point, lanes over the nodes of both pieces
    for (int j = warp; j < FUZZ_A_TERMS; j += kWarps) {
        const float cq = cospif((j + 0.5f) / (2.0f * FUZZ_A_TERMS));
        const float mu = cq * cq;
        const float st = sqrtf(fmaxf(0.0f, 1.0f - mu * mu)), split = asinf(mu);
        KSum acc;
        for (int q = lane; q < 2 * kNA; q += 32) {
            const int g = q % kNA;
            const bool outer = q >= kNA;
            const float lo = outer ? split : 0.0f, hi = outer ? 0.5f * PT_PI_F : split;
            const float th = 0.5f * (hi + lo) + 0.5f * (hi - lo) * fa_x[g], w = 0.5f * (hi - lo) * fa_w[g];
            float sn, ct;
            sincosf(th, &sn, &ct);
            const float b = mu * ct, a = st * sn;
            float inner;
            if (b >= a) {
                inner = 2.0f * PT_PI_F * b;
            } else {
                const float c = -b / a;
                inner = 2.0f * a * sqrtf(fmaxf(0.0f, 1.0f - c * c)) + 2.0f * b * acosf(c);
            }
            acc.add(w * (charlie_D_s2(sn * sn, alpha) * sn * inner));
        }
        const float s = warp_ksum(acc);
        if (lane == 0) a_val[j] = s;
    }
    __syncthreads();
    if (t < FUZZ_A_TERMS) c_a[t] = cheb_coef(a_val, FUZZ_A_TERMS, t);
    __syncthreads();

    // E at the Chebyshev points of x = 2 mu^(1/4) - 1: mu^(1/4) = cos^2(pi (j + 1/2) / 64);
    // one warp per point
    for (int j = warp; j < FUZZ_E_TERMS; j += kWarps) {
        const float cq = cospif((j + 0.5f) / (2.0f * FUZZ_E_TERMS));
        const float q = cq * cq, q2 = q * q;
        const float mu_o = q2 * q2;
        const float so = sqrtf(fmaxf(0.0f, 1.0f - mu_o * mu_o));
        const float a_o = cheb_smem(c_a, FUZZ_A_TERMS, 2.0f * mu_o - 1.0f);
        KSum acc;
        float lo = 0.0f, hi = fmaxf(mu_o, kFloor);
        while (lo < 1.0f) {
            const float t0 = acosf(hi), t1 = acosf(lo);
            const float cut = fminf(PT_PI_F, 8.0f * (mu_o + hi));
            if (lane < kNT) {
                const float th = 0.5f * (t0 + t1) + 0.5f * (t1 - t0) * ft_x[lane];
                float si, mi;
                sincosf(th, &si, &mi);
                const float a_i = cheb_smem(c_a, FUZZ_A_TERMS, 2.0f * mi - 1.0f);
                piece_mu[warp][lane] = mi;
                piece_s[warp][lane] = si;
                // polar weight times mu_i sin(theta_i) / (4 (A_i mu_o + A_o mu_i - mu_i mu_o))
                piece_k[warp][lane] = 0.5f * (t1 - t0) * ft_w[lane] * mi * si /
                                      (4.0f * (a_i * mu_o + a_o * mi - mi * mu_o));
            }
            __syncwarp();
            for (int part = 0; part < 2; ++part) {
                const float p0 = part == 0 ? 0.0f : PT_PI_F - cut, p1 = part == 0 ? PT_PI_F - cut : PT_PI_F;
                if (!(p1 > p0)) continue;
                for (int idx = lane; idx < kNT * kNP; idx += 32) {
                    const int i = idx / kNP, p = idx % kNP;
                    const float ph = 0.5f * (p0 + p1) + 0.5f * (p1 - p0) * fp_x[p];
                    const float wp = 0.5f * (p1 - p0) * fp_w[p];
                    float sp, cp;
                    sincosf(ph, &sp, &cp);
                    const float mi = piece_mu[warp][i], si = piece_s[warp][i];
                    const float hx = si * cp + so, hy = si * sp, hz = mi + mu_o;
                    const float hxy = hx * hx + hy * hy;
                    const float s2 = hxy / (hxy + hz * hz);
                    acc.add(wp * piece_k[warp][i] * charlie_D_s2(s2, alpha));
                }
            }
            __syncwarp();
            lo = hi;
            hi = fminf(4.0f * lo, 1.0f);
        }
        const float s = 2.0f * warp_ksum(acc);
        if (lane == 0) e_val[j] = s;
    }
    __syncthreads();
    if (t < FUZZ_A_TERMS) o[FUZZ_HEAD + t] = c_a[t];
    if (t < FUZZ_E_TERMS) o[FUZZ_HEAD + FUZZ_A_TERMS + t] = cheb_coef(e_val, FUZZ_E_TERMS, t);
}

}  // namespace

pt_status pt_fuzz_series(const float* raw_materials, uint32_t n, float* out, cudaStream_t st) {
    if (n == 0) return PT_OK;
    PT_LAUNCH(k_fuzz_series, n, kThreads, 0, st, raw_materials, n, out);
    PT_CUDA_TRY(cudaGetLastError());
    return PT_OK;
}
