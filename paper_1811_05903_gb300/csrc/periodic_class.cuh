// Box tests that sort the images of a tile pair for the periodic pair term
// (Sec. 2.2, Eq. 5, cut at |x_i - x_j - nL| < 2.6 L, and the quasi-periodic
// leading term), shared by the symmetric
// far-field kernel and the per-target kernel so that both make exactly the same
// decision for every (tile pair, image).
//
// Coordinates are in box units (L = 1) with tile centres on a grid that makes
// c_I - c_J - n exact in FP32; then the image n of (I, J) and the image -n of
// (J, I) have separations of exactly opposite sign, and every test below is
// symmetric under that exchange.
#pragma once

#include <cuda_runtime.h>

namespace steps {

constexpr int kPerImages = 343;      // candidate images |n_c| <= 3 (a term needs |n_c| < 3.6)
constexpr int kPerZeroImage = 171;   // index of n = 0; index k = 49 (nx + 3) + 7 (ny + 3) + (nz + 3)

enum PeriodicClass { kPerNone = 0, kPerInside = 1, kPerStraddle = 2, kPerSoft = 3 };

__device__ __forceinline__ void periodic_image_of(int k, int &nx, int &ny, int &nz) {
    nx = k / 49 - 3;
    ny = (k / 7) % 7 - 3;
    nz = k % 7 - 3;
}

// Class of image n of the tile pair (I, J), box units.  ci/cj: (centre, hmax),
// ei/ej: (half extents, mass).  kPerSoft: some pair may lie within h_i + h_j
// (or I == J and n = 0: the self pairs); kPerInside: every pair is Newtonian
// and inside the cut sphere; kPerStraddle: every pair Newtonian, some may lie
// outside the sphere; kPerNone: no pair inside the sphere.  The extents carry a
// margin of 1e-5 (the FP32 tests round at ~1e-7).  gap2 receives the squared
// distance between the two boxes (a lower bound on r^2 of every pair).
__device__ __forceinline__ int periodic_image_class(const float4 ci, const float4 ei, const float4 cj,
                                                    const float4 ej, int nx, int ny, int nz, bool self,
                                                    float *gap2_out) {
    const float up = 1.0f + 0x1p-18f, dn = 1.0f - 0x1p-18f;
    const float mg = 1e-5f;
    const float cut2 = 2.6f * 2.6f;
    // exact: the centres lie on a common grid and n is a small integer
    const float sx = __fsub_rn(__fsub_rn(ci.x, cj.x), (float)nx);
    const float sy = __fsub_rn(__fsub_rn(ci.y, cj.y), (float)ny);
    const float sz = __fsub_rn(__fsub_rn(ci.z, cj.z), (float)nz);
    const float wx = __fadd_rn(__fmul_rn(__fadd_rn(ei.x, ej.x), up), mg);
    const float wy = __fadd_rn(__fmul_rn(__fadd_rn(ei.y, ej.y), up), mg);
    const float wz = __fadd_rn(__fmul_rn(__fadd_rn(ei.z, ej.z), up), mg);
    const float ax = fabsf(sx), ay = fabsf(sy), az = fabsf(sz);
    const float gx = fmaxf(0.f, __fsub_rn(ax, wx)), gy = fmaxf(0.f, __fsub_rn(ay, wy)),
                gz = fmaxf(0.f, __fsub_rn(az, wz));
    const float fx = __fadd_rn(ax, wx), fy = __fadd_rn(ay, wy), fz = __fadd_rn(az, wz);
    const float gap2 = __fmaf_rn(gz, gz, __fmaf_rn(gy, gy, __fmul_rn(gx, gx)));
    const float far2 = __fmaf_rn(fz, fz, __fmaf_rn(fy, fy, __fmul_rn(fx, fx)));
    *gap2_out = gap2;
    if (!(gap2 < __fmul_rn(cut2, up))) return kPerNone;
    const float hs = __fmul_rn(__fadd_rn(ci.w, cj.w), up);
    if ((self && nx == 0 && ny == 0 && nz == 0) || gap2 <= __fmul_rn(hs, hs)) return kPerSoft;
    return far2 < __fmul_rn(cut2, dn) ? kPerInside : kPerStraddle;
}

// Quasi-periodic sum: the single image with x_i - x_j - nL in [-L/2, L/2)^3;
// candidates |n_c| <= 1 (positions wrapped into the box), index
// k = 9 (nx + 1) + 3 (ny + 1) + (nz + 1).
constexpr int kQuasiImages = 27;
constexpr int kQuasiZeroImage = 13;

__device__ __forceinline__ void quasi_image_of(int k, int &nx, int &ny, int &nz) {
    nx = k / 9 - 1;
    ny = (k / 3) % 3 - 1;
    nz = k % 3 - 1;
}

// Class of image n of the tile pair (I, J) for the quasi-periodic sum, box
// units: kPerInside when every pair has |d_c| < 1/2 in every component,
// kPerStraddle when some may, kPerNone when none can, kPerSoft as above.  The
// same margins as the cut sum's tests; symmetric under the exchange.
__device__ __forceinline__ int quasi_image_class(const float4 ci, const float4 ei, const float4 cj, const float4 ej,
                                                 int nx, int ny, int nz, bool self, float *gap2_out) {
    const float up = 1.0f + 0x1p-18f, dn = 1.0f - 0x1p-18f;
    const float mg = 1e-5f;
    const float sx = __fsub_rn(__fsub_rn(ci.x, cj.x), (float)nx);
    const float sy = __fsub_rn(__fsub_rn(ci.y, cj.y), (float)ny);
    const float sz = __fsub_rn(__fsub_rn(ci.z, cj.z), (float)nz);
    const float wx = __fadd_rn(__fmul_rn(__fadd_rn(ei.x, ej.x), up), mg);
    const float wy = __fadd_rn(__fmul_rn(__fadd_rn(ei.y, ej.y), up), mg);
    const float wz = __fadd_rn(__fmul_rn(__fadd_rn(ei.z, ej.z), up), mg);
    const float ax = fabsf(sx), ay = fabsf(sy), az = fabsf(sz);
    const float gx = fmaxf(0.f, __fsub_rn(ax, wx)), gy = fmaxf(0.f, __fsub_rn(ay, wy)),
                gz = fmaxf(0.f, __fsub_rn(az, wz));
    const float gap2 = __fmaf_rn(gz, gz, __fmaf_rn(gy, gy, __fmul_rn(gx, gx)));
    *gap2_out = gap2;
    const float half_up = __fmul_rn(0.5f, up), half_dn = __fmul_rn(0.5f, dn);
    if (!(gx < half_up && gy < half_up && gz < half_up)) return kPerNone;
    const float hs = __fmul_rn(__fadd_rn(ci.w, cj.w), up);
    if ((self && nx == 0 && ny == 0 && nz == 0) || gap2 <= __fmul_rn(hs, hs)) return kPerSoft;
    return (__fadd_rn(ax, wx) < half_dn && __fadd_rn(ay, wy) < half_dn && __fadd_rn(az, wz) < half_dn)
               ? kPerInside
               : kPerStraddle;
}

namespace {

// Whether the term (i, j, n) counts, decided in FP64 from the FP64 positions as the
// definition states it (no contraction).
__device__ __noinline__ bool include_f64(double xi, double yi, double zi, double xj, double yj, double zj, int nx,
                                        int ny, int nz, double L, int images) {
    const double d0x = __dsub_rn(xi, xj), d0y = __dsub_rn(yi, yj), d0z = __dsub_rn(zi, zj);
    if (images == 1) {
        return floor(__dadd_rn(__ddiv_rn(d0x, L), 0.5)) == (double)nx &&
               floor(__dadd_rn(__ddiv_rn(d0y, L), 0.5)) == (double)ny &&
               floor(__dadd_rn(__ddiv_rn(d0z, L), 0.5)) == (double)nz;
    }
    const double dx = __dsub_rn(d0x, __dmul_rn((double)nx, L));
    const double dy = __dsub_rn(d0y, __dmul_rn((double)ny, L));
    const double dz = __dsub_rn(d0z, __dmul_rn((double)nz, L));
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    const double cut = __dmul_rn(2.6, L);
    return r2 < __dmul_rn(cut, cut);
}

}  // namespace

}  // namespace steps
