// pat_lut.cu -- the lookup tables of the paper's LUT variant of the
// cylinder's arc integral (Sec. 4.2.2): E~(s, m) = E(arcsin s, m) and
// F~(s, m) = F(arcsin s, m) on the power-law grid of Eq. (LUT_sampling) in s
// and in m, evaluated once per plan on the device in FP64 and stored per cell
// for float-float bilinear interpolation (layout in LutDev).
//
// With x = 1 - s^2 and y = 1 - m s^2 (the incomplete integrals in Carlson's
// symmetric form, DLMF 19.25.5 and 19.25.9):
//   F~ = s R_F(x, y, 1),   E~ = F~ - (m / 3) s^3 R_D(x, y, 1).
// x and y are formed from the complements 1 - s and 1 - m, which are exact
// for the nodes (s, m >= 1/2), so the logarithmic corner (s, m) -> (1, 1)
// keeps full relative precision.
#include <algorithm>

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

// One thread per table node: (E~, F~) in FP64 into V [ns][nm].
__global__ void lut_nodes_kernel(int ns, int nm, double2 *__restrict__ V)
{
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
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
    V[id] = make_double2(E, F);
}

__device__ __forceinline__ float2 split_d(double v)
{
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

// One thread per cell (i, j) < (ns - 1, nm - 1): the corner value in
// float-float and the bilinear differences in FP32 (layout in LutDev); the
// first threads also write the node arrays.
__global__ void lut_cells_kernel(int ns, int nm, const double2 *__restrict__ V, float4 *__restrict__ A,
                                 float4 *__restrict__ B, float2 *__restrict__ C, float2 *__restrict__ gs,
                                 float *__restrict__ hs, float2 *__restrict__ gm, float *__restrict__ hm)
{
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id < ns) {
        const int n = (int)id;
        gs[n] = split_d(lut_grid(n, ns));
        hs[n] = n < ns - 1 ? (float)(1.0 / (lut_grid(n + 1, ns) - lut_grid(n, ns))) : 0.f;
    }
    if (id < nm) {
        const int n = (int)id;
        gm[n] = split_d(lut_grid(n, nm));
        hm[n] = n < nm - 1 ? (float)(1.0 / (lut_grid(n + 1, nm) - lut_grid(n, nm))) : 0.f;
    }
    const long long ncell = (long long)(ns - 1) * (nm - 1);
    if (id >= ncell) return;
    const int i = (int)(id / (nm - 1)), j = (int)(id % (nm - 1));
    const double2 v00 = V[(size_t)i * nm + j], v01 = V[(size_t)i * nm + j + 1];
    const double2 v10 = V[(size_t)(i + 1) * nm + j], v11 = V[(size_t)(i + 1) * nm + j + 1];
    const float2 e = split_d(v00.x), f = split_d(v00.y);
    A[id] = make_float4(e.x, e.y, (float)(v01.x - v00.x), (float)(v10.x - v00.x));
    B[id] = make_float4((float)((v11.x - v10.x) - (v01.x - v00.x)), f.x, f.y, (float)(v01.y - v00.y));
    C[id] = make_float2((float)(v10.y - v00.y), (float)((v11.y - v10.y) - (v01.y - v00.y)));
}

size_t lut_bytes(int ns, int nm)
{
    const size_t cells = (size_t)(ns - 1) * (nm - 1);
    return cells * (sizeof(float4) * 2 + sizeof(float2)) + (size_t)(ns + nm) * (sizeof(float2) + sizeof(float));
}

cudaError_t launch_lut_tables(int ns, int nm, void *buf, double2 *scratch, LutDev &L, cudaStream_t st)
{
    const size_t cells = (size_t)(ns - 1) * (nm - 1);
    char *p = (char *)buf;
    float4 *A = (float4 *)p;
    float4 *B = A + cells;
    float2 *C = (float2 *)(B + cells);
    float2 *gs = C + cells, *gm = gs + ns;
    float *hs = (float *)(gm + nm), *hm = hs + ns;
    L.A = A;
    L.B = B;
    L.C = C;
    L.gs = gs;
    L.gm = gm;
    L.hs = hs;
    L.hm = hm;
    L.ns = ns;
    L.nm = nm;
    const double top = lut_grid(ns - 1, ns); // the same 1 - eps for both axes
    const float th = (float)top;
    L.top = make_float2(th, (float)(top - (double)th));
    const long long n = (long long)ns * nm;
    lut_nodes_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ns, nm, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long m = std::max((long long)cells, (long long)std::max(ns, nm));
    lut_cells_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(ns, nm, scratch, A, B, C, gs, hs, gm, hm);
    return cudaGetLastError();
}

} // namespace pat
