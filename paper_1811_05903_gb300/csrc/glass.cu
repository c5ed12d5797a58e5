// Spherical-glass initial conditions (Sec. 3.1): particles placed shell by
// shell in the compactified space and mapped back to real space.
//
// Compactification (Eq. 14-15): real-space radius r <-> angle
// omega = 2 arctan(r / D_s) on the 3-sphere of diameter D_s.  The 3-sphere's
// volume element is (D_s/2)^3 sin^2(omega) sin(theta) d omega d theta d phi,
// so the compact volume inside omega is (pi D_s^3 / 8) F(omega) with
// F(omega) = 2 omega - sin 2 omega, the function of Eq. 18.
//
// Two slicings of the compactified space:
//  * constant delta-omega: n_radial shells of equal width in omega from
//    omega_c = 2 arctan(r_c / D_s) to omega_max = 2 arctan(R_sim / D_s); the
//    ball r < r_c is one volume of N_inner = floor((4 pi/3) r_c^3 rho_bar /
//    m_inner) equal-mass particles (Eq. 17), m_inner being the particle mass of
//    the first shell (the mass is continuous at r_c), placed uniformly in real
//    space;
//  * constant compact volume: edges with F(omega_i) = i F(omega_max) / n_radial
//    (Eq. 18), found by bisection.
// Each shell gets n_shell particles uniform in its compact volume (omega from
// the sin^2 density by bisection on F, direction uniform on the sphere) at
// Eq. 15's real-space position, with mass rho_bar V_shell / n_shell (Eq. 16,
// V_shell the real-space shell volume).  The random numbers are the caller's.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "steps_internal.h"

namespace steps {
namespace {

// F(omega) = 2 omega - sin 2 omega (compact volume inside omega, in units of pi D_s^3 / 8)
__host__ __device__ inline double compact_F(double w) { return 2.0 * w - sin(2.0 * w); }

struct Layout {
    std::vector<double> edges;   // [n_radial + 1] omega
    std::vector<double> m_shell; // [n_radial]
    int64_t n_inner = 0;
    double m_inner = 0.0;
    int64_t n_total = 0;
};

steps_status check_spec(const steps_glass_spec *s) {
    if (!s) {
        set_error("spec is NULL");
        return STEPS_EINVAL;
    }
    const bool finite = std::isfinite(s->D_s) && std::isfinite(s->R_sim) && std::isfinite(s->rho_bar);
    if (!finite || !(s->D_s > 0.0) || !(s->R_sim > 0.0) || !(s->rho_bar > 0.0) || s->n_radial < 1 ||
        s->n_shell < 1) {
        set_error("D_s, R_sim and rho_bar must be finite and > 0, n_radial and n_shell >= 1");
        return STEPS_EINVAL;
    }
    if (s->scheme != STEPS_GLASS_CONST_DOMEGA && s->scheme != STEPS_GLASS_CONST_VOLUME) {
        set_error("unknown glass scheme %d", s->scheme);
        return STEPS_EINVAL;
    }
    if (s->scheme == STEPS_GLASS_CONST_DOMEGA && !(s->r_c > 0.0 && s->r_c < s->R_sim)) {
        set_error("r_c must lie in (0, R_sim) for the constant delta-omega scheme");
        return STEPS_EINVAL;
    }
    return STEPS_OK;
}

steps_status make_layout(const steps_glass_spec *s, Layout *L) {
    STEPS_TRY(check_spec(s));
    const int nr = s->n_radial;
    const double w_max = 2.0 * std::atan(s->R_sim / s->D_s);
    L->edges.assign(nr + 1, 0.0);
    if (s->scheme == STEPS_GLASS_CONST_DOMEGA) {
        const double w_c = 2.0 * std::atan(s->r_c / s->D_s);
        for (int i = 0; i <= nr; ++i) L->edges[i] = w_c + (w_max - w_c) * (double)i / (double)nr;
    } else {
        const double F_max = compact_F(w_max);
        for (int i = 1; i < nr; ++i) {
            const double target = F_max * (double)i / (double)nr;
            double a = 0.0, b = w_max;
            for (int it = 0; it < 200; ++it) {
                const double mid = 0.5 * (a + b);
                if (mid <= a || mid >= b) break;
                if (compact_F(mid) < target) a = mid; else b = mid;
            }
            L->edges[i] = 0.5 * (a + b);
        }
        L->edges[nr] = w_max;
    }
    L->m_shell.assign(nr, 0.0);
    for (int i = 0; i < nr; ++i) {
        const double r0 = s->D_s * std::tan(0.5 * L->edges[i]);
        const double r1 = s->D_s * std::tan(0.5 * L->edges[i + 1]);
        L->m_shell[i] = s->rho_bar * (4.0 * M_PI / 3.0 * (r1 * r1 * r1 - r0 * r0 * r0)) / (double)s->n_shell;
    }
    L->n_inner = 0;
    L->m_inner = 0.0;
    if (s->scheme == STEPS_GLASS_CONST_DOMEGA) {
        L->m_inner = L->m_shell[0];
        L->n_inner = (int64_t)std::floor(4.0 * M_PI / 3.0 * s->r_c * s->r_c * s->r_c * s->rho_bar / L->m_inner);
    }
    L->n_total = L->n_inner + (int64_t)nr * s->n_shell;
    return STEPS_OK;
}

// One thread per particle: the inner ball's particles first, then n_shell per
// shell in shell order.  u[k] = (u_omega, u_cos, u_phi).
__global__ void glass_place_kernel(int64_t n, int64_t n_inner, int64_t n_shell, double r_c, double D_s,
                                   double m_inner, const double *__restrict__ edges,
                                   const double *__restrict__ m_shell, const double *__restrict__ u,
                                   double *__restrict__ pos, double *__restrict__ mass) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double u0 = u[3 * k], u1 = u[3 * k + 1], u2 = u[3 * k + 2];
    double radius, m;
    if (k < n_inner) {
        radius = r_c * cbrt(u0);
        m = m_inner;
    } else {
        const int64_t sh = (k - n_inner) / n_shell;
        const double lo = edges[sh], hi = edges[sh + 1];
        const double target = compact_F(lo) + u0 * (compact_F(hi) - compact_F(lo));
        double a = lo, b = hi;
        for (int it = 0; it < 200; ++it) {
            const double mid = 0.5 * (a + b);
            if (mid <= a || mid >= b) break;
            if (compact_F(mid) < target) a = mid; else b = mid;
        }
        radius = D_s * tan(0.25 * (a + b));  // Eq. 15 radial part at omega = (a + b) / 2
        m = m_shell[sh];
    }
    const double ct = 1.0 - 2.0 * u1;
    const double stheta = sqrt(fmax(0.0, 1.0 - ct * ct));
    const double phi = 2.0 * M_PI * u2;
    pos[3 * k] = radius * stheta * cos(phi);
    pos[3 * k + 1] = radius * stheta * sin(phi);
    pos[3 * k + 2] = radius * ct;
    mass[k] = m;
}

}  // namespace
}  // namespace steps

using namespace steps;

extern "C" steps_status steps_glass_layout(const steps_glass_spec *spec, int64_t *n_total, int64_t *n_inner,
                                           double *m_inner, double *omega_edges, double *shell_mass) {
    Layout L;
    STEPS_TRY(make_layout(spec, &L));
    if (n_total) *n_total = L.n_total;
    if (n_inner) *n_inner = L.n_inner;
    if (m_inner) *m_inner = L.m_inner;
    if (omega_edges)
        for (size_t i = 0; i < L.edges.size(); ++i) omega_edges[i] = L.edges[i];
    if (shell_mass)
        for (size_t i = 0; i < L.m_shell.size(); ++i) shell_mass[i] = L.m_shell[i];
    return STEPS_OK;
}

extern "C" steps_status steps_glass_place(const steps_glass_spec *spec, int64_t n, const double *u, double *pos,
                                          double *mass, void *cuda_stream) {
    Layout L;
    STEPS_TRY(make_layout(spec, &L));
    if (n != L.n_total) {
        set_error("n = %lld but the layout holds %lld particles", (long long)n, (long long)L.n_total);
        return STEPS_EINVAL;
    }
    if (!u || !pos || !mass) {
        set_error("u, pos and mass are required");
        return STEPS_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int nr = spec->n_radial;
    const size_t bytes = sizeof(double) * ((size_t)(2 * nr + 1) + 7 * (size_t)n) + 64;
    void *mem = nullptr;
    STEPS_TRY(counted_malloc(&mem, bytes));
    double *d_edges = static_cast<double *>(mem);
    double *d_mass_shell = d_edges + (nr + 1);
    double *d_u = d_mass_shell + nr;
    double *d_pos = d_u + 3 * n;
    double *d_mass = d_pos + 3 * n;
    steps_status status = STEPS_OK;
    cudaError_t e = cudaMemcpyAsync(d_edges, L.edges.data(), sizeof(double) * (nr + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_mass_shell, L.m_shell.data(), sizeof(double) * nr, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_u, u, sizeof(double) * 3 * n, cudaMemcpyDefault, st);
    if (e == cudaSuccess) {
        glass_place_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, L.n_inner, spec->n_shell, spec->r_c,
                                                                        spec->D_s, L.m_inner, d_edges,
                                                                        d_mass_shell, d_u, d_pos, d_mass);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(pos, d_pos, sizeof(double) * 3 * n, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(mass, d_mass, sizeof(double) * n, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) status = cuda_status(e, "steps_glass_place");
    cudaStreamSynchronize(st);
    counted_free(mem, bytes);
    return status;
}
