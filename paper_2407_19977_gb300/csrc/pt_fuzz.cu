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
//      starts to dip below the horizon of w (theta_m = asin(mu)), 48 Gauss points a piece;
//   E: 32 terms in x = 2 sqrt(mu) - 1 (E behaves like mu log mu at grazing), from E at the
//      32 Chebyshev points, each a 2-D integral: mu_i over the pieces [0, mu_o], [mu_o, 8 mu_o],
//      [8 mu_o, 64 mu_o], ... (the integrand turns over at mu_i ~ mu_o, and D has a kink at
//      mu_i = mu_o), 16 Gauss points a piece, the azimuth over [0, pi] (the integrand is even)
//      with 48 Gauss points; A(mu_i) from its series.
#include <cmath>

#include "pt_device.cuh"
#include "pt_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kGA = 48;      // Gauss points per piece of the A integral
constexpr int kGM = 16;      // per piece of the mu_i integral of E
constexpr int kGP = 48;      // over the azimuth of E
constexpr int kRatio = 8;    // growth of the mu_i pieces
constexpr int kMaxPieces = 16;   // mu_o >= 3.6e-7 at the Chebyshev points needs 9
constexpr double kPi = 3.14159265358979323846;

// node j of the n-point Gauss-Legendre rule on [-1, 1]: a root of P_n by Newton's method
// from cos(pi (j + 3/4) / (n + 1/2)); weight 2 / ((1 - x^2) P_n'(x)^2)
__device__ void gauss_node(int n, int j, double* x_out, double* w_out) {
    double x = cos(kPi * (j + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 64; ++it) {
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (x * p1 - p0) / (x * x - 1.0);
        const double dx = p1 / dp;
        x -= dx;
        if (fabs(dx) < 1e-15) break;
    }
    *x_out = x;
    *w_out = 2.0 / ((1.0 - x * x) * dp * dp);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
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

// one material per CTA; raw rows of PT_OPENPBR_FLOATS floats; out FUZZ_FLOATS per row (the
// head fw, fc[3], a, then the A and E series; zeros for a row without fuzz)
__global__ void __launch_bounds__(kThreads) k_fuzz_series(const float* __restrict__ raw, uint32_t n,
                                                          float* __restrict__ out) {
    __shared__ double ga_x[kGA], ga_w[kGA], gm_x[kGM], gm_w[kGM], gp_x[kGP], gp_w[kGP];
    __shared__ float a_val[FUZZ_A_TERMS], e_val[FUZZ_E_TERMS], c_a[FUZZ_A_TERMS];
    __shared__ float gp_c[kGP], gp_s[kGP];   // cos, sin of the azimuth nodes
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
    if (t < kGA) gauss_node(kGA, t, &ga_x[t], &ga_w[t]);
    else if (t < kGA + kGM) gauss_node(kGM, t - kGA, &gm_x[t - kGA], &gm_w[t - kGA]);
    else if (t < kGA + kGM + kGP) gauss_node(kGP, t - kGA - kGM, &gp_x[t - kGA - kGM], &gp_w[t - kGA - kGM]);
    __syncthreads();
    if (t < kGP) {
        const double ph = 0.5 * kPi * (1.0 + gp_x[t]);
        gp_c[t] = (float)cos(ph);
        gp_s[t] = (float)sin(ph);
    }
    __syncthreads();

    // A at the Chebyshev points mu_j = (1 + cos(pi (j + 1/2) / 16)) / 2: one warp per point
    for (int j = warp; j < FUZZ_A_TERMS; j += kWarps) {
        const double mu = 0.5 * (1.0 + cos(kPi * (j + 0.5) / FUZZ_A_TERMS));
        const double st = sqrt(fmax(0.0, 1.0 - mu * mu)), split = asin(mu);
        double acc = 0.0;
        for (int q = lane; q < 2 * kGA; q += 32) {
            const int g = q % kGA;
            const bool outer = q >= kGA;
            const double lo = outer ? split : 0.0, hi = outer ? 0.5 * kPi : split;
            const double th = 0.5 * (hi + lo) + 0.5 * (hi - lo) * ga_x[g], w = 0.5 * (hi - lo) * ga_w[g];
            const float ct = (float)cos(th), sn = (float)sin(th);
            const float b = (float)mu * ct, a = (float)st * sn;
            float inner;
            if (b >= a) {
                inner = 2.0f * PT_PI_F * b;
            } else {
                const float c = -b / a;
                inner = 2.0f * a * sqrtf(fmaxf(0.0f, 1.0f - c * c)) + 2.0f * b * acosf(c);
            }
            acc += w * (double)(sheen_D(ct, alpha) * sn * inner);
        }
        acc = warp_sum(acc);
        if (lane == 0) a_val[j] = (float)acc;
    }
    __syncthreads();
    if (t < FUZZ_A_TERMS) {
        double c = 0.0;
        for (int j = 0; j < FUZZ_A_TERMS; ++j) c += a_val[j] * cos(kPi * t * (j + 0.5) / FUZZ_A_TERMS);
        c *= 2.0 / FUZZ_A_TERMS;
        if (t == 0) c *= 0.5;
        c_a[t] = (float)c;
    }
    __syncthreads();

    // E at the Chebyshev points of x = 2 sqrt(mu) - 1: one warp per point
    for (int j = warp; j < FUZZ_E_TERMS; j += kWarps) {
        const double sq = 0.5 * (1.0 + cos(kPi * (j + 0.5) / FUZZ_E_TERMS));
        const float mu_o = (float)(sq * sq);
        const float so = sqrtf(fmaxf(0.0f, 1.0f - mu_o * mu_o));
        const float a_o = cheb_smem(c_a, FUZZ_A_TERMS, 2.0f * mu_o - 1.0f);
        double acc = 0.0;
        double lo = 0.0, hi = mu_o;
        for (int piece = 0; piece < kMaxPieces && lo < 1.0; ++piece) {
            for (int i = 0; i < kGM; ++i) {
                const double mi_d = 0.5 * (hi + lo) + 0.5 * (hi - lo) * gm_x[i];
                const double wm = 0.5 * (hi - lo) * gm_w[i];
                const float mi = (float)mi_d, si = sqrtf(fmaxf(0.0f, 1.0f - mi * mi));
                const float a_i = cheb_smem(c_a, FUZZ_A_TERMS, 2.0f * mi - 1.0f);
                const float den = 4.0f * (a_i * mu_o + a_o * mi - mi * mu_o);
                for (int p = lane; p < kGP; p += 32) {
                    const double wp = 0.5 * kPi * gp_w[p];
                    const float hx = si * gp_c[p] + so, hy = si * gp_s[p], hz = mi + mu_o;
                    const float cz = hz * rsqrtf(hx * hx + hy * hy + hz * hz);
                    acc += wm * wp * (double)(sheen_D(cz, alpha) * mi / den);
                }
            }
            lo = hi;
            hi = fmin(hi * kRatio, 1.0);
        }
        acc = 2.0 * warp_sum(acc);
        if (lane == 0) e_val[j] = (float)acc;
    }
    __syncthreads();
    if (t < FUZZ_A_TERMS) o[FUZZ_HEAD + t] = c_a[t];
    if (t < FUZZ_E_TERMS) {
        double c = 0.0;
        for (int j = 0; j < FUZZ_E_TERMS; ++j) c += e_val[j] * cos(kPi * t * (j + 0.5) / FUZZ_E_TERMS);
        c *= 2.0 / FUZZ_E_TERMS;
        if (t == 0) c *= 0.5;
        o[FUZZ_HEAD + FUZZ_A_TERMS + t] = (float)c;
    }
}

}  // namespace

pt_status pt_fuzz_series(const float* raw_materials, uint32_t n, float* out, cudaStream_t st) {
    if (n == 0) return PT_OK;
    PT_LAUNCH(k_fuzz_series, n, kThreads, 0, st, raw_materials, n, out);
    PT_CUDA_TRY(cudaGetLastError());
    return PT_OK;
}
