// pat_lut.cu -- the lookup tables of the paper's LUT variant of the
// cylinder's arc integral (Sec. 4.2.2): E~(s, m) = E(arcsin s, m) and
// F~(s, m) = F(arcsin s, m) on the power-law grid of Eq. (LUT_sampling) in s
// and in m, built once per plan on the device in FP64.
//
// With x = 1 - s^2 and y = 1 - m s^2 (the incomplete integrals in Carlson's
// symmetric form, DLMF 19.25.5 and 19.25.9):
//   F~ = s R_F(x, y, 1),   E~ = F~ - (m / 3) s^3 R_D(x, y, 1).
// x and y are formed from the complements 1 - s and 1 - m, which are exact
// for the nodes (s, m >= 1/2), so the logarithmic corner (s, m) -> (1, 1)
// keeps full relative precision.
#include "pat_kernels.cuh"

namespace pat {

// Carlson's R_F by the duplication theorem (DLMF 19.26.18): each step maps
// (x, y, z) to ((x + l) / 4, ...), l = sqrt(x y) + sqrt(y z) + sqrt(z x),
// which leaves R_F unchanged and pulls the arguments together; once their
// relative spread around the mean A is below 2e-3, the fifth-order
// expansion of DLMF 19.36.1 in the elementary symmetric functions E2, E3 of
// the deviations X = 1 - x/A (X + Y + Z = 0) is exact to about 1e-17.
__device__ double lut_rf(double x, double y, double z)
{
    for (int it = 0; it < 64; ++it) {
        const double A = (x + y + z) / 3.0;
        const double X = 1.0 - x / A, Y = 1.0 - y / A, Z = -(X + Y);
        if (fmax(fabs(X), fmax(fabs(Y), fabs(Z))) < 2e-3) {
            const double E2 = X * Y + Y * Z + Z * X, E3 = X * Y * Z;
            const double ser = 1.0 - E2 / 10.0 + E3 / 14.0 + E2 * E2 / 24.0 - 3.0 * E2 * E3 / 44.0;
            return ser / sqrt(A);
        }
        const double rx = sqrt(x), ry = sqrt(y), rz = sqrt(z);
        const double l = rx * ry + ry * rz + rz * rx;
        x = 0.25 * (x + l);
        y = 0.25 * (y + l);
        z = 0.25 * (z + l);
    }
    return __longlong_as_double(0x7ff8000000000000LL); // not converged: NaN
}

// Carlson's R_D by duplication (DLMF 19.26.20): each step adds
// 3 / (4^k sqrt(z) (z + l)); the remainder is 4^-k A^(-3/2) times the
// expansion of DLMF 19.36.2, with E2..E5 the elementary symmetric functions
// of the five deviations (X, Y, Z, Z, Z), X = 1 - x/A, A = (x + y + 3 z) / 5.
__device__ double lut_rd(double x, double y, double z)
{
    double sum = 0.0, f = 1.0;
    for (int it = 0; it < 64; ++it) {
        const double A = (x + y + 3.0 * z) / 5.0;
        const double X = 1.0 - x / A, Y = 1.0 - y / A, Z = 1.0 - z / A;
        if (fmax(fabs(X), fmax(fabs(Y), fabs(Z))) < 2e-3) {
            const double Z2 = Z * Z, Z3 = Z2 * Z;
            const double E2 = X * Y + 3.0 * Z * (X + Y) + 3.0 * Z2;
            const double E3 = 3.0 * X * Y * Z + 3.0 * Z2 * (X + Y) + Z3;
            const double E4 = 3.0 * X * Y * Z2 + Z3 * (X + Y);
            const double E5 = X * Y * Z3;
            const double ser = 1.0 - 3.0 * E2 / 14.0 + E3 / 6.0 + 9.0 * E2 * E2 / 88.0 - 3.0 * E4 / 22.0 -
                               9.0 * E2 * E3 / 52.0 + 3.0 * E5 / 26.0;
            return sum + f * ser / (A * sqrt(A));
        }
        const double rx = sqrt(x), ry = sqrt(y), rz = sqrt(z);
        const double l = rx * ry + ry * rz + rz * rx;
        sum += 3.0 * f / (rz * (z + l));
        f *= 0.25;
        x = 0.25 * (x + l);
        y = 0.25 * (y + l);
        z = 0.25 * (z + l);
    }
    return __longlong_as_double(0x7ff8000000000000LL);
}

// One thread per table node; the first threads also write the node arrays.
__global__ void lut_tables_kernel(int ns, int nm, double2 *__restrict__ T, double *__restrict__ gs,
                                  double *__restrict__ hs, double *__restrict__ gm, double *__restrict__ hm)
{
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id < ns) {
        const int n = (int)id;
        gs[n] = lut_grid(n, ns);
        hs[n] = n < ns - 1 ? 1.0 / (lut_grid(n + 1, ns) - lut_grid(n, ns)) : 0.0;
    }
    if (id < nm) {
        const int n = (int)id;
        gm[n] = lut_grid(n, nm);
        hm[n] = n < nm - 1 ? 1.0 / (lut_grid(n + 1, nm) - lut_grid(n, nm)) : 0.0;
    }
    if (id >= (long long)ns * nm) return;
    const int i = (int)(id / nm), j = (int)(id % nm);
    const double s = lut_grid(i, ns), m = lut_grid(j, nm);
    double E = 0.0, F = 0.0;
    if (s > 0.0) {
        const double s2 = s * s;
        const double x = (1.0 - s) * (1.0 + s);
        const double y = fma(1.0 - m, s2, x);
        F = s * lut_rf(x, y, 1.0);
        E = F - (m / 3.0) * s2 * s * lut_rd(x, y, 1.0);
    }
    T[id] = make_double2(E, F);
}

cudaError_t launch_lut_tables(int ns, int nm, double2 *T, double *gs, double *hs, double *gm, double *hm,
                              cudaStream_t st)
{
    const long long n = (long long)ns * nm;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    lut_tables_kernel<<<blocks, 256, 0, st>>>(ns, nm, T, gs, hs, gm, hm);
    return cudaGetLastError();
}

} // namespace pat
