// Point-force source (Eq. ex_homo): the displacement it radiates into a homogeneous medium, Eq. ex_anal,
// and its time derivative, sampled on a regular grid as initial data for the decomposition.
#include <algorithm>
#include <cmath>

#include "fga_internal.cuh"

namespace fga {
namespace {

// Gauss-Legendre rule of order 8 on [-1, 1]: the roots of P_8 by Newton's method from Chebyshev
// guesses, weights 2 / ((1 - x^2) P_8'(x)^2)
struct GaussLegendre8 {
    double x[8], w[8];
};

GaussLegendre8 make_gl8() {
    GaussLegendre8 g{};
    const int n = 8;
    for (int i = 0; i < n; i++) {
        double x = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = x;  // P_0, P_1
            for (int k = 2; k <= n; k++) {
                const double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);  // P_n'(x)
            const double dx = p1 / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; k++) {
                const double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
        }
        g.x[i] = x;
        g.w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    return g;
}

const GaussLegendre8 &gl8() {
    static const GaussLegendre8 g = make_gl8();
    return g;
}

struct SourceDev {
    double x0[3], d[3];
    double rho, cp, cs, om, T0, sigma;
    double panel;   // longest quadrature panel (s)
};

// s(t) = cos(omega (t + T0)) exp(-(t + T0)^2 / sigma^2) and s'(t)
__device__ __forceinline__ void stf(const SourceDev &S, double t, double &s, double &ds) {
    const double a = t + S.T0;
    const double e = exp(-(a / S.sigma) * (a / S.sigma));
    double sn, cs;
    sincos(S.om * a, &sn, &cs);
    s = cs * e;
    ds = (-S.om * sn - 2.0 * a / (S.sigma * S.sigma) * cs) * e;
}

// per grid point: u (and du/dt) of Eq. ex_anal; the near-field integral int_a^b tau s(t - tau) dtau
// (a = r/c_p, b = r/c_s) by composite Gauss-Legendre quadrature, its time derivative through
// a s(t - a) - b s(t - b) + int_a^b s(t - tau) dtau (integration by parts); panels whose every node
// lies more than 8.6 sigma from the pulse centre (envelope below e^-74) are skipped
__global__ void __launch_bounds__(128) point_force_kernel(SourceDev S, GaussLegendre8 G, int n0, int n1, int n2,
                                                          double3 y0, double3 dy, double t, double2 *__restrict__ u,
                                                          double2 *__restrict__ v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = (int64_t)n0 * n1 * n2;
    if (i >= n) return;
    const int i2 = (int)(i % n2), i1 = (int)((i / n2) % n1), i0 = (int)(i / ((int64_t)n1 * n2));
    const double X[3] = {y0.x + i0 * dy.x - S.x0[0], y0.y + i1 * dy.y - S.x0[1], y0.z + i2 * dy.z - S.x0[2]};
    const double r = sqrt(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
    const double scale = 1.0 + fabs(S.x0[0]) + fabs(S.x0[1]) + fabs(S.x0[2]);
    double ou[3] = {0.0, 0.0, 0.0}, ov[3] = {0.0, 0.0, 0.0};
    if (r > 1e-12 * scale) {
        const double g[3] = {X[0] / r, X[1] / r, X[2] / r};
        const double gd = g[0] * S.d[0] + g[1] * S.d[1] + g[2] * S.d[2];
        const double a = r / S.cp, b = r / S.cs;
        double sp, dsp, ss, dss;
        stf(S, t - a, sp, dsp);
        stf(S, t - b, ss, dss);
        // near-field integrals
        double I = 0.0, J = 0.0;  // int tau s(t - tau), int s(t - tau)
        const int npan = (int)ceil((b - a) / S.panel);
        const double L = (b - a) / npan;
        const double lim = 8.6 * S.sigma;
        for (int pi = 0; pi < npan; pi++) {
            const double lo = a + pi * L, hi = lo + L;
            // w = t + T0 - tau over the panel
            const double wlo = t + S.T0 - hi, whi = t + S.T0 - lo;
            if (wlo > lim || whi < -lim) continue;
            const double c = 0.5 * (lo + hi), h = 0.5 * L;
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const double tau = c + h * G.x[q];
                double s, ds;
                stf(S, t - tau, s, ds);
                I += G.w[q] * h * tau * s;
                J += G.w[q] * h * s;
            }
        }
        const double It = a * sp - b * ss + J;
        const double kp = 1.0 / (4.0 * M_PI * S.rho * S.cp * S.cp * r);
        const double ks = 1.0 / (4.0 * M_PI * S.rho * S.cs * S.cs * r);
        const double kn = 1.0 / (4.0 * M_PI * S.rho * r * r * r);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const double gg = g[c] * gd;
            ou[c] = gg * kp * sp + (S.d[c] - gg) * ks * ss + (3.0 * gg - S.d[c]) * kn * I;
            ov[c] = gg * kp * dsp + (S.d[c] - gg) * ks * dss + (3.0 * gg - S.d[c]) * kn * It;
        }
    }
    if (u)
        for (int c = 0; c < 3; c++) u[3 * i + c] = make_double2(ou[c], 0.0);
    if (v)
        for (int c = 0; c < 3; c++) v[3 * i + c] = make_double2(ov[c], 0.0);
}

}  // namespace
}  // namespace fga

using namespace fga;

extern "C" fga_status fga_point_force_field(const fga_point_force *src, const int ny[3], const double y0[3],
                                            const double dy[3], double t, void *u_out, void *v_out,
                                            fga_stream_t s_) {
    cudaStream_t s = (cudaStream_t)s_;
    FGA_CHECK(src && ny && y0 && dy, "fga_point_force_field: NULL argument");
    FGA_CHECK(u_out || v_out, "fga_point_force_field: both outputs are NULL");
    FGA_CHECK(std::isfinite(t), "fga_point_force_field: t is not finite");
    FGA_CHECK(src->rho > 0 && src->cs > 0 && src->cp > src->cs && std::isfinite(src->cp),
              "fga_point_force_field: need rho > 0 and 0 < c_s < c_p");
    FGA_CHECK(src->sigma > 0 && std::isfinite(src->sigma) && src->f >= 0 && std::isfinite(src->f) &&
                  std::isfinite(src->T0),
              "fga_point_force_field: need sigma > 0, f >= 0 and a finite T0");
    int64_t n = 1;
    for (int a = 0; a < 3; a++) {
        FGA_CHECK(ny[a] >= 1 && dy[a] > 0 && std::isfinite(y0[a]) && std::isfinite(dy[a]),
                  "fga_point_force_field: need ny >= 1 and dy > 0 per axis");
        FGA_CHECK(std::isfinite(src->x0[a]) && std::isfinite(src->force[a]), "fga_point_force_field: bad x0 or force");
        n *= ny[a];
    }
    FGA_CHECK(n < ((int64_t)1 << 37), "fga_point_force_field: grid too large");
    SourceDev S;
    for (int a = 0; a < 3; a++) {
        S.x0[a] = src->x0[a];
        S.d[a] = src->force[a];
    }
    S.rho = src->rho;
    S.cp = src->cp;
    S.cs = src->cs;
    S.om = 2.0 * M_PI * src->f;
    S.T0 = src->T0;
    S.sigma = src->sigma;
    // panels of at most 1/8 of a period and 1/4 of sigma
    S.panel = src->sigma / 4.0;
    if (src->f > 0) S.panel = std::min(S.panel, 1.0 / (8.0 * src->f));
    const GaussLegendre8 G = gl8();
    const unsigned blocks = (unsigned)((n + 127) / 128);
    {
        ProfScope ps(P_DECOMP, s);
        point_force_kernel<<<blocks, 128, 0, s>>>(S, G, ny[0], ny[1], ny[2], make_double3(y0[0], y0[1], y0[2]),
                                                  make_double3(dy[0], dy[1], dy[2]), t, static_cast<double2 *>(u_out),
                                                  static_cast<double2 *>(v_out));
    }
    FGA_CUDA(cudaGetLastError());
    return FGA_OK;
}
