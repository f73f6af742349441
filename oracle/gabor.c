/*
 * gabor.c - CPU oracle of the orientation and confidence maps the paper extracts with Gabor filters
 * (Sec. 3.1: O in R^{H x W x 2}, C in [0, 1]^{H x W}); the paper gives no filter parameters, so the
 * bank, the response and the confidence below are readings (listed in the design notes).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or load this file: only
 * the tests, the smoke check and the benchmark's CPU-baseline leg use it.  It shares no code,
 * header, table or constant with the CUDA library.
 *
 *  bank   n_theta orientations theta_k = k pi / n_theta; on the (2r+1) x (2r+1) window of offsets
 *         (u right, v down): along a = u cos theta + v sin theta, across b = -u sin theta + v cos
 *         theta, envelope exp(-a^2 / (2 sa^2) - b^2 / (2 sb^2)); even kernel envelope x
 *         cos(2 pi b / lambda) minus its window mean, odd kernel envelope x sin(2 pi b / lambda);
 *         both rounded to bfloat16 (round to nearest even), the precision the GPU multiplies in;
 *  input  the image rounded to bfloat16, zero outside;
 *  F_k    sqrt(e_k^2 + o_k^2), e_k / o_k the window correlations (sums in double);
 *  theta  theta_k* with k* the largest F_k, the first on ties;
 *  flag   set where the index is not determined at single precision: the two largest F lie within
 *         m = 2 (2r+1) 2^-22 max_k (S_e,k + S_o,k) + 2^-16 F_k*, where S_e,k, S_o,k are the sums of
 *         the absolute products of the two correlations.  The first term bounds twice the error of
 *         F_k when each correlation is accumulated in FP32 one window row at a time (the row's exact
 *         bf16 products added to the running sum with a relative error of at most 2^-22 of the
 *         absolute sum so far: 2r+1 such steps); the second covers F^2 formed in FP32 and compared
 *         at a 16-bit relative resolution;
 *  C      1 - mean_k F_k / F_k* (0 where every F is 0).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static float bf16_round(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return x;   /* inf / nan unchanged */
    u = (u + 0x7fffu + ((u >> 16) & 1u)) & 0xffff0000u;
    float y;
    memcpy(&y, &u, 4);
    return y;
}

float or_bf16(float x) { return bf16_round(x); }

/* out: n_theta x 2 x (2r+1)^2 floats (even then odd kernel of each orientation, row v, column u). */
void or_gabor_bank(int n_theta, int r, double sa, double sb, double lambda, float* out) {
    const int w = 2 * r + 1, n = w * w;
    double* ev = (double*)malloc(sizeof(double) * n);
    for (int k = 0; k < n_theta; k++) {
        const double th = 3.14159265358979323846 * k / n_theta, c = cos(th), s = sin(th);
        double mean = 0.0;
        for (int v = -r; v <= r; v++)
            for (int u = -r; u <= r; u++) {
                const double a = u * c + v * s, b = -u * s + v * c;
                const double env = exp(-a * a / (2.0 * sa * sa) - b * b / (2.0 * sb * sb));
                const int q = (v + r) * w + (u + r);
                ev[q] = env * cos(2.0 * 3.14159265358979323846 * b / lambda);
                mean += ev[q];
                out[(size_t)(2 * k + 1) * n + q] = bf16_round((float)(env * sin(2.0 * 3.14159265358979323846 * b / lambda)));
            }
        mean /= n;
        for (int q = 0; q < n; q++) out[(size_t)(2 * k) * n + q] = bf16_round((float)(ev[q] - mean));
    }
    free(ev);
}

/* Orientation index, angle, confidence and flag at the listed pixels of one H x W image. */
void or_gabor_pixels(const float* img, int H, int W, int n_theta, int r, const float* bank, long long n_idx,
                     const long long* idx, int32_t* kbest, float* theta, float* conf, uint8_t* flag) {
    const int w = 2 * r + 1, n = w * w;
    double* F = (double*)malloc(sizeof(double) * n_theta);
    for (long long q = 0; q < n_idx; q++) {
        const long long pix = idx[q];
        const int y = (int)(pix / W), x = (int)(pix % W);
        double best = -1.0, second = -1.0, sum = 0.0, smax = 0.0;
        int kb = 0;
        for (int k = 0; k < n_theta; k++) {
            double e = 0.0, o = 0.0, abs_sum = 0.0;
            for (int v = -r; v <= r; v++) {
                const int yy = y + v;
                if (yy < 0 || yy >= H) continue;
                for (int u = -r; u <= r; u++) {
                    const int xx = x + u;
                    if (xx < 0 || xx >= W) continue;
                    const double iv = bf16_round(img[(size_t)yy * W + xx]);
                    const int t = (v + r) * w + (u + r);
                    e += bank[(size_t)(2 * k) * n + t] * iv;
                    o += bank[(size_t)(2 * k + 1) * n + t] * iv;
                    abs_sum += fabs(bank[(size_t)(2 * k) * n + t] * iv) + fabs(bank[(size_t)(2 * k + 1) * n + t] * iv);
                }
            }
            F[k] = sqrt(e * e + o * o);
            if (abs_sum > smax) smax = abs_sum;
            sum += F[k];
            if (F[k] > best) {
                second = best;
                best = F[k];
                kb = k;
            } else if (F[k] > second) {
                second = F[k];
            }
        }
        kbest[q] = kb;
        theta[q] = (float)(3.14159265358979323846 * kb / n_theta);
        conf[q] = best > 0.0 ? (float)(1.0 - sum / n_theta / best) : 0.0f;
        const double margin = 2.0 * ldexp((double)w, -22) * smax + ldexp(best, -16);
        flag[q] = (uint8_t)(second >= 0.0 && best - second <= margin);
    }
    free(F);
}
