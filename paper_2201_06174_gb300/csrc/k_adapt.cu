// K3a: the paper's adaptive weight update (LMS, NLMS, RLS; Eq. 4 and the adaptive scheme around it)
// run as the sequential filters they are: one recursion per chain, in FP64, over the voxels in the
// order inline sections (y) outermost, then x, then t.  Chains are independent blocks of `sections`
// inline sections (the re-adaptation after every N sections the paper allows); sections = 0 is one
// chain over the whole volume.  One warp per chain: the lanes stage the normalised maps
// x_m = (S_m - lo_m) / (hi_m - lo_m) and the desired value d of the next 32 steps in shared memory
// while lane 0 runs the FP64 recursion over the current 32 (a single FP64 chain; FP64 throughput on
// this part is low, so no lane repeats it).
//   LMS:  W += mu e x
//   NLMS: W += mu e x / (eps + |x|^2)
//   RLS:  k = P x / (lambda + x'Px);  W += k e;  P = (P - k x'P) / lambda,  P0 = I/delta
// with e = d - W.x; W0 = (1/3, 1/3, 1/3) for LMS and NLMS, 0 for RLS.
#include "sal_internal.cuh"

namespace sal {
namespace {

enum : int { ADAPT_LMS = 0, ADAPT_NLMS = 1, ADAPT_RLS = 2 };

__global__ void __launch_bounds__(32)
k3_adapt(const float* __restrict__ S3, const float* __restrict__ D, int T, int X, int Y, int method, double mu,
         double eps, double lambda, double delta, int sec, const float* __restrict__ norm, float* __restrict__ W_out,
         float* __restrict__ err2) {
    __shared__ double s_x[2][4][32];   // two chunks of 32 steps: x_t, x_x, x_y, d
    const long long NV = (long long)T * X * Y;
    const int lane = threadIdx.x;
    const int y_begin = blockIdx.x * sec, y_end = min(Y, y_begin + sec);
    const long long steps = (long long)(y_end - y_begin) * X * T;
    const long long first = (long long)y_begin * X * T;   // index of this chain's first step in filter order
    const double lo0 = norm[0], lo1 = norm[1], lo2 = norm[2];
    const double iv0 = norm[3], iv1 = norm[4], iv2 = norm[5];
    const double inv_lambda = 1.0 / lambda;
    // the recursion state lives in lane 0 (one FP64 chain; the other lanes stage the next chunk)
    double w0, w1, w2;
    if (method == ADAPT_RLS) w0 = w1 = w2 = 0.0;
    else w0 = w1 = w2 = 1.0 / 3.0;
    double P[3][3] = {{1.0 / delta, 0.0, 0.0}, {0.0, 1.0 / delta, 0.0}, {0.0, 0.0, 1.0 / delta}};
    auto stage = [&](long long base, int buf) {
        const long long s = base + lane;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, dv = 0.0;
        if (s < steps) {
            const int t = (int)(s % T), x = (int)((s / T) % X), y = y_begin + (int)(s / ((long long)T * X));
            const long long p = ((long long)t * X + x) * Y + y;
            a0 = ((double)__ldg(S3 + p) - lo0) * iv0;
            a1 = ((double)__ldg(S3 + NV + p) - lo1) * iv1;
            a2 = ((double)__ldg(S3 + 2 * NV + p) - lo2) * iv2;
            dv = (double)__ldg(D + p);
        }
        s_x[buf][0][lane] = a0;
        s_x[buf][1][lane] = a1;
        s_x[buf][2][lane] = a2;
        s_x[buf][3][lane] = dv;
    };
    stage(0, 0);
    __syncwarp();
    int buf = 0;
    for (long long base = 0; base < steps; base += 32, buf ^= 1) {
        if (base + 32 < steps) stage(base + 32, buf ^ 1);   // the next chunk, while lane 0 runs this one
        if (lane == 0) {
            const int cnt = steps - base < 32 ? (int)(steps - base) : 32;
            for (int i = 0; i < cnt; ++i) {
                const double x0 = s_x[buf][0][i], x1 = s_x[buf][1][i], x2 = s_x[buf][2][i], d = s_x[buf][3][i];
                const double e = d - (w0 * x0 + w1 * x1 + w2 * x2);
                if (err2) err2[first + base + i] = (float)(e * e);
                if (method == ADAPT_LMS) {
                    w0 += mu * e * x0;
                    w1 += mu * e * x1;
                    w2 += mu * e * x2;
                } else if (method == ADAPT_NLMS) {
                    const double g = mu * e / (eps + (x0 * x0 + x1 * x1 + x2 * x2));
                    w0 += g * x0;
                    w1 += g * x1;
                    w2 += g * x2;
                } else {
                    double Px[3], xP[3];
#pragma unroll
                    for (int r = 0; r < 3; ++r) {
                        Px[r] = P[r][0] * x0 + P[r][1] * x1 + P[r][2] * x2;
                        xP[r] = x0 * P[0][r] + x1 * P[1][r] + x2 * P[2][r];
                    }
                    const double inv_den = 1.0 / (lambda + x0 * Px[0] + x1 * Px[1] + x2 * Px[2]);
                    const double k0 = Px[0] * inv_den, k1 = Px[1] * inv_den, k2 = Px[2] * inv_den;
                    w0 += k0 * e;
                    w1 += k1 * e;
                    w2 += k2 * e;
                    const double kk[3] = {k0, k1, k2};
#pragma unroll
                    for (int r = 0; r < 3; ++r)
#pragma unroll
                        for (int c = 0; c < 3; ++c) P[r][c] = (P[r][c] - kk[r] * xP[c]) * inv_lambda;
                }
            }
        }
        __syncwarp();
    }
    if (lane == 0) {
        W_out[blockIdx.x * 3 + 0] = (float)w0;
        W_out[blockIdx.x * 3 + 1] = (float)w1;
        W_out[blockIdx.x * 3 + 2] = (float)w2;
    }
}

}  // namespace

cudaError_t adapt_launch(const float* S3, const float* D, int T, int X, int Y, int method, double mu, double eps,
                         double lambda, double delta, int sections, const float* norm, float* W_out, float* err2,
                         cudaStream_t s) {
    const int sec = sections > 0 ? sections : Y;
    const int blocks = (Y + sec - 1) / sec;
    k3_adapt<<<blocks, 32, 0, s>>>(S3, D, T, X, Y, method, mu, eps, lambda, delta, sec, norm, W_out, err2);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace sal
