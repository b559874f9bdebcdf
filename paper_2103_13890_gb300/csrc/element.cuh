// Element arithmetic of the Q1 residuals with the 2^d-point Gauss rule.
//
// The element integrals are the ones of the problem definitions (Sec. 3 and
// the nonlinear-diffusion problems): for a Q1 element with nodal values u_abc
//   R_abc = sum_q w_q [ c(u_q) grad u_q . grad phi_abc(q) (+ source term) ]
// with Gauss points 1/2 +- 1/(2 sqrt 3) per direction.
//
// Evaluation order (exact reformulation, rounding differs from a quadrature
// loop):  a 1D Q1 function at the two Gauss points is m +- A delta with
// m = (u0+u1)/2, delta = (u1-u0)/2 and A = 1/sqrt 3, and its derivative is
// 2 delta / h.  So the nodal values are first turned into "modal"
// coefficients by sum/difference butterflies in each direction, the values and
// gradients at all Gauss points follow from 2-point butterflies of the scaled
// modes, and the test-function side is the transpose of the same chain.  In
// 3D this costs 164 floating-point operations per element for nonlinear
// diffusion (a direct quadrature loop needs ~500), which matters because FP64
// throughput on GB300 is ~1/61 of FP32.
#pragma once

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace jfnk {

// a b + c (the compiler contracts it to one FMA for float and double; the
// packed two-element type of the FP32 kernels overloads it)
template <typename T>
__host__ __device__ __forceinline__ T madd(T a, T b, T c) {
    return a * b + c;
}

// 2-point butterfly over two sign variables, forward:
//   out[i][j] = v00 + s_i v10 + s_j v01 + s_i s_j v11,  s_0 = -1, s_1 = +1
template <typename T>
__host__ __device__ __forceinline__ void h2_fwd(T v00, T v10, T v01, T v11, T out[2][2]) {
    T t0p = v00 + v01, t0m = v00 - v01;
    T t1p = v10 + v11, t1m = v10 - v11;
    out[1][1] = t0p + t1p;
    out[0][1] = t0p - t1p;
    out[1][0] = t0m + t1m;
    out[0][0] = t0m - t1m;
}

// transpose: w_pq = sum_{i,j} s_i^p s_j^q F[i][j]
template <typename T>
__host__ __device__ __forceinline__ void h2_adj(const T F[2][2], T& w00, T& w10, T& w01, T& w11) {
    T S0 = F[1][0] + F[0][0], S1 = F[1][1] + F[0][1];
    T D0 = F[1][0] - F[0][0], D1 = F[1][1] - F[0][1];
    w00 = S1 + S0;
    w01 = S1 - S0;
    w10 = D1 + D0;
    w11 = D1 - D0;
}

// ---------------------------------------------------------------------------
// 3D nonlinear diffusion element.
//   u[8]: nodal values, index a + 2b + 4c for offsets (a, b, c) in (x, y, z)
//   kap:  per-element coefficient (1 for the plain problem)
//   r[8]: sum_q (1/ (3h/16)) * w_q * kap (1+u_q^2) grad u_q . grad phi_abc(q),
//         i.e. the element residual divided by 3h/16, which the caller applies
//         once per node.
// ---------------------------------------------------------------------------
// Middle of the element for its modal inputs: a_pq and b_pq are the x/y
// butterflies of the nodal values on the element's lower (c = 0) and upper
// (c = 1) z face (p: x mode, q: y mode; mode 0 = sum, mode 1 = difference), and
// the outputs are the test-function modes R_pqr (R_000 = 0) before the
// transposed butterflies.  elem_nd3 below is forward butterflies + this +
// transposed butterflies; the z-marching kernels share the face butterflies of
// neighbouring elements and call this directly (same operations, same order).
template <typename T, bool KAPPA>
__host__ __device__ __forceinline__ void elem_nd3_mid(T a00, T a01, T a10, T a11, T b00, T b01, T b10, T b11,
                                                      T kap, T& R001, T& R010, T& R011, T& R100, T& R101,
                                                      T& R110, T& R111) {
    const T A1 = T(0.57735026918962576451);   // 1/sqrt(3)
    const T A2 = T(0.33333333333333333333);   // 1/3
    const T A3 = T(0.19245008972987525484);   // 1/(3 sqrt 3)
    // S_pqr = M'_pqr A^(p+q+r) / 8  (8 ops)
    // (A^k / 8 is exact in either precision: the scaling by 2^-3 does not round)
    const T A1s = T(0.57735026918962576451 * 0.125), A2s = T(0.33333333333333333333 * 0.125),
            A3s = T(0.19245008972987525484 * 0.125);
    T S000 = (a00 + b00) * T(0.125);
    T S001 = (b00 - a00) * A1s;
    T S010 = (a01 + b01) * A1s;
    T S011 = (b01 - a01) * A2s;
    T S100 = (a10 + b10) * A1s;
    T S101 = (b10 - a10) * A2s;
    T S110 = (a11 + b11) * A2s;
    T S111 = (b11 - a11) * A3s;
    // values and (scaled) gradients at the Gauss points (40 ops)
    T P0[2][2], GX[2][2], GY[2][2], GZ[2][2];
    h2_fwd(S000, S010, S001, S011, P0);  // [sy][sz]
    h2_fwd(S100, S110, S101, S111, GX);  // [sy][sz]  d/dx = 2/(hA) GX
    h2_fwd(S010, S110, S011, S111, GY);  // [sx][sz]
    h2_fwd(S001, S101, S011, S111, GZ);  // [sx][sy]
    // coefficient c = kap (1 + u^2) at the 8 points, index [sx][sy][sz]
    T c[2][2][2];
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            T up = P0[j][k] + GX[j][k];
            T um = P0[j][k] - GX[j][k];
            if (KAPPA) {
                c[1][j][k] = madd(kap * up, up, kap);
                c[0][j][k] = madd(kap * um, um, kap);
            } else {
                c[1][j][k] = madd(up, up, T(1));
                c[0][j][k] = madd(um, um, T(1));
            }
        }
    // sum the flux over the direction its gradient factor does not depend on
    T FX[2][2], FY[2][2], FZ[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            FX[i][j] = GX[i][j] * (c[1][i][j] + c[0][i][j]);  // [sy][sz]
            FY[i][j] = GY[i][j] * (c[i][1][j] + c[i][0][j]);  // [sx][sz]
            FZ[i][j] = GZ[i][j] * (c[i][j][1] + c[i][j][0]);  // [sx][sy]
        }
    T X00, X10, X01, X11, Y00, Y10, Y01, Y11, Z00, Z10, Z01, Z11;
    h2_adj(FX, X00, X10, X01, X11);  // X_qr
    h2_adj(FY, Y00, Y10, Y01, Y11);  // Y_pr
    h2_adj(FZ, Z00, Z10, Z01, Z11);  // Z_pq
    // test-function modes, scaled by A^(p+q+r) (12 ops)
    R100 = X00 * A1;
    R010 = Y00 * A1;
    R001 = Z00 * A1;
    R110 = (X10 + Y10) * A2;
    R101 = (X01 + Z10) * A2;
    R011 = (Y01 + Z01) * A2;
    R111 = (X11 + Y11 + Z11) * A3;
}

template <typename T, bool KAPPA>
__host__ __device__ __forceinline__ void elem_nd3(const T u[8], T kap, T r[8]) {
    // modal transform M' = T' (x) T' (x) T' u, T' = [[1,1],[-1,1]]  (24 ops)
    T p0 = u[0] + u[1], q0 = u[1] - u[0];
    T p1 = u[2] + u[3], q1 = u[3] - u[2];
    T p2 = u[4] + u[5], q2 = u[5] - u[4];
    T p3 = u[6] + u[7], q3 = u[7] - u[6];
    T a00 = p0 + p1, a01 = p1 - p0, b00 = p2 + p3, b01 = p3 - p2;  // x-mode 0
    T a10 = q0 + q1, a11 = q1 - q0, b10 = q2 + q3, b11 = q3 - q2;  // x-mode 1
    T R001, R010, R011, R100, R101, R110, R111;
    elem_nd3_mid<T, KAPPA>(a00, a01, a10, a11, b00, b01, b10, b11, kap, R001, R010, R011, R100, R101, R110, R111);
    // transpose of the modal transform (R000 = 0)  (24 ops)
    // z pass: (mode r) -> (c)
    T e00_0 = -R001, e00_1 = R001;            // (p,q) = (0,0)
    T e01_0 = R010 - R011, e01_1 = R010 + R011;  // (0,1)
    T e10_0 = R100 - R101, e10_1 = R100 + R101;  // (1,0)
    T e11_0 = R110 - R111, e11_1 = R110 + R111;  // (1,1)
    // y pass: (mode q) -> (b)
    T f0_00 = e00_0 - e01_0, f0_10 = e00_0 + e01_0;  // p=0, (b,c)=(0,0),(1,0)
    T f0_01 = e00_1 - e01_1, f0_11 = e00_1 + e01_1;  // p=0, (0,1),(1,1)
    T f1_00 = e10_0 - e11_0, f1_10 = e10_0 + e11_0;
    T f1_01 = e10_1 - e11_1, f1_11 = e10_1 + e11_1;
    // x pass: (mode p) -> (a)
    r[0] = f0_00 - f1_00; r[1] = f0_00 + f1_00;
    r[2] = f0_10 - f1_10; r[3] = f0_10 + f1_10;
    r[4] = f0_01 - f1_01; r[5] = f0_01 + f1_01;
    r[6] = f0_11 - f1_11; r[7] = f0_11 + f1_11;
}

// ---------------------------------------------------------------------------
// 3D vector-Jacobian product of the coefficient problem (adjoint).
//   F_i = sum_e kap_e int_e (1+u^2) grad u . grad phi_i - int phi_i, so for a
//   (boundary-masked) w:
//   (J^T w)_b  = kap int_e (1+u^2) grad w . grad phi_b + 2 u (grad u . grad w) phi_b
//   (dF/dkap_e)^T w = int_e (1+u^2) grad u . grad w
// u[8], w[8] nodal values (index a + 2b + 4c).  r[8] receives (J^T w)_b / (3h/16),
// dk receives (dF/dkap_e)^T w / (3h/2).  The first term has the residual's
// structure with grad w in the flux; the second is a mass-like term whose test
// side is the transpose of the 3D Gauss-point interpolation.
// ---------------------------------------------------------------------------
template <typename T>
__host__ __device__ __forceinline__ void modal_scaled3(const T u[8], T S[8]) {
    // S[p + 2q + 4r] = M'_pqr A^(p+q+r) / 8 with M' = T' (x) T' (x) T' u
    const T A1 = T(0.57735026918962576451);
    const T A2 = T(0.33333333333333333333);
    const T A3 = T(0.19245008972987525484);
    T p0 = u[0] + u[1], q0 = u[1] - u[0];
    T p1 = u[2] + u[3], q1 = u[3] - u[2];
    T p2 = u[4] + u[5], q2 = u[5] - u[4];
    T p3 = u[6] + u[7], q3 = u[7] - u[6];
    T a00 = p0 + p1, a01 = p1 - p0, b00 = p2 + p3, b01 = p3 - p2;
    T a10 = q0 + q1, a11 = q1 - q0, b10 = q2 + q3, b11 = q3 - q2;
    S[0] = (a00 + b00) * T(0.125);
    S[4] = (b00 - a00) * (A1 * T(0.125));
    S[2] = (a01 + b01) * (A1 * T(0.125));
    S[6] = (b01 - a01) * (A2 * T(0.125));
    S[1] = (a10 + b10) * (A1 * T(0.125));
    S[5] = (b10 - a10) * (A2 * T(0.125));
    S[3] = (a11 + b11) * (A2 * T(0.125));
    S[7] = (b11 - a11) * (A3 * T(0.125));
}

template <typename T>
__host__ __device__ __forceinline__ void elem_vjp3(const T u[8], const T w[8], T kap, T r[8], T& dk) {
    const T A1 = T(0.57735026918962576451);
    const T A2 = T(0.33333333333333333333);
    const T A3 = T(0.19245008972987525484);
    T Su[8], Sw[8];
    modal_scaled3(u, Su);
    modal_scaled3(w, Sw);
    T P0[2][2], GXu[2][2], GYu[2][2], GZu[2][2], GXw[2][2], GYw[2][2], GZw[2][2];
    h2_fwd(Su[0], Su[2], Su[4], Su[6], P0);   // [sy][sz]
    h2_fwd(Su[1], Su[3], Su[5], Su[7], GXu);  // [sy][sz]
    h2_fwd(Su[2], Su[3], Su[6], Su[7], GYu);  // [sx][sz]
    h2_fwd(Su[4], Su[5], Su[6], Su[7], GZu);  // [sx][sy]
    h2_fwd(Sw[1], Sw[3], Sw[5], Sw[7], GXw);
    h2_fwd(Sw[2], Sw[3], Sw[6], Sw[7], GYw);
    h2_fwd(Sw[4], Sw[5], Sw[6], Sw[7], GZw);
    T c[2][2][2], src[2][2][2];
    T dks = T(0);
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const T uq = i ? P0[j][k] + GXu[j][k] : P0[j][k] - GXu[j][k];
                const T g = uq * uq + T(1);
                const T dot = GXu[j][k] * GXw[j][k] + GYu[i][k] * GYw[i][k] + GZu[i][j] * GZw[i][j];
                c[i][j][k] = kap * g;
                src[i][j][k] = uq * dot;
                dks += g * dot;
            }
    dk = dks;
    T FX[2][2], FY[2][2], FZ[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            FX[i][j] = GXw[i][j] * (c[1][i][j] + c[0][i][j]);
            FY[i][j] = GYw[i][j] * (c[i][1][j] + c[i][0][j]);
            FZ[i][j] = GZw[i][j] * (c[i][j][1] + c[i][j][0]);
        }
    T X00, X10, X01, X11, Y00, Y10, Y01, Y11, Z00, Z10, Z01, Z11;
    h2_adj(FX, X00, X10, X01, X11);
    h2_adj(FY, Y00, Y10, Y01, Y11);
    h2_adj(FZ, Z00, Z10, Z01, Z11);
    // E_pqr = sum over the 8 points of s_x^p s_y^q s_z^r src
    T Ez0[2][2], Ez1[2][2];  // [sx][sy] sums / differences over sz
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            Ez0[i][j] = src[i][j][1] + src[i][j][0];
            Ez1[i][j] = src[i][j][1] - src[i][j][0];
        }
    T E000, E100, E010, E110, E001, E101, E011, E111;
    h2_adj(Ez0, E000, E100, E010, E110);
    h2_adj(Ez1, E001, E101, E011, E111);
    const T k2 = kap + kap;
    const T R000 = k2 * E000;
    const T R100 = (X00 + k2 * E100) * A1, R010 = (Y00 + k2 * E010) * A1, R001 = (Z00 + k2 * E001) * A1;
    const T R110 = (X10 + Y10 + k2 * E110) * A2;
    const T R101 = (X01 + Z10 + k2 * E101) * A2;
    const T R011 = (Y01 + Z01 + k2 * E011) * A2;
    const T R111 = (X11 + Y11 + Z11 + k2 * E111) * A3;
    T e00_0 = R000 - R001, e00_1 = R000 + R001;
    T e01_0 = R010 - R011, e01_1 = R010 + R011;
    T e10_0 = R100 - R101, e10_1 = R100 + R101;
    T e11_0 = R110 - R111, e11_1 = R110 + R111;
    T f0_00 = e00_0 - e01_0, f0_10 = e00_0 + e01_0;
    T f0_01 = e00_1 - e01_1, f0_11 = e00_1 + e01_1;
    T f1_00 = e10_0 - e11_0, f1_10 = e10_0 + e11_0;
    T f1_01 = e10_1 - e11_1, f1_11 = e10_1 + e11_1;
    r[0] = f0_00 - f1_00; r[1] = f0_00 + f1_00;
    r[2] = f0_10 - f1_10; r[3] = f0_10 + f1_10;
    r[4] = f0_01 - f1_01; r[5] = f0_01 + f1_01;
    r[6] = f0_11 - f1_11; r[7] = f0_11 + f1_11;
}

// ---------------------------------------------------------------------------
// 2D Bratu element (Sec. 3).
//   u[4]: nodal values, index a + 2b
//   lh:   lambda h^2 / 16
//   r[4]: int_e grad u_h . grad phi_ab - lambda exp(u_h) phi_ab   (exact scale)
// With M' = T' (x) T' u the gradient part in modal form is
// (0, M'_10/4, M'_01/4, M'_11/6) and the source part is
// -(lambda h^2/16) A^(p+q) sum_q s_x^p s_y^q exp(u_q).
// ---------------------------------------------------------------------------
template <typename T>
__host__ __device__ __forceinline__ T exp_t(T x);
template <>
__host__ __device__ __forceinline__ double exp_t<double>(double x) { return exp(x); }
template <>
__host__ __device__ __forceinline__ float exp_t<float>(float x) { return expf(x); }

template <typename T>
__host__ __device__ __forceinline__ void elem_bratu2(const T u[4], T lh, T r[4]) {
    const T A1 = T(0.57735026918962576451);
    const T A2 = T(0.33333333333333333333);
    T p0 = u[0] + u[1], q0 = u[1] - u[0];
    T p1 = u[2] + u[3], q1 = u[3] - u[2];
    T M00 = p0 + p1, M01 = p1 - p0, M10 = q0 + q1, M11 = q1 - q0;
    T S00 = M00 * T(0.25), S10 = M10 * (A1 * T(0.25));
    T S01 = M01 * (A1 * T(0.25)), S11 = M11 * (A2 * T(0.25));
    T U[2][2];  // [sx][sy]
    h2_fwd(S00, S10, S01, S11, U);
    T E[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) E[i][j] = exp_t<T>(U[i][j]);
    T E00, E10, E01, E11;
    h2_adj(E, E00, E10, E01, E11);
    T la1 = lh * A1, la2 = lh * A2;
    T R00 = -lh * E00;
    T R10 = M10 * T(0.25) - la1 * E10;
    T R01 = M01 * T(0.25) - la1 * E01;
    T R11 = M11 * T(0.16666666666666666667) - la2 * E11;
    // transpose of the modal transform
    T g0_0 = R00 - R01, g0_1 = R00 + R01;  // p=0, b=0/1
    T g1_0 = R10 - R11, g1_1 = R10 + R11;  // p=1
    r[0] = g0_0 - g1_0; r[1] = g0_0 + g1_0;
    r[2] = g0_1 - g1_1; r[3] = g0_1 + g1_1;
}

// ---------------------------------------------------------------------------
// 2D minimal-surface element (Sec. 3, "Minimal Surface").
//   u[4]:   nodal values, index a + 2b
//   inv_h2: 1/h^2
//   r[4]:   int_e grad u_h . grad phi_ab / sqrt(1 + |grad u_h|^2)   (exact scale)
// With the modes M of elem_bratu2, h grad u_h at the Gauss point (sx, sy) is
//   (M10/2 + sy (A/2) M11,  M01/2 + sx (A/2) M11),
// the x component depends on sy only and the y component on sx only.  With
// X_q = c_q Gx_q / 4, Y_q = c_q Gy_q / 4 (c = 1/sqrt(1+|grad u|^2), weights 1/4)
// the test-function side is r_ab = s_a P1 + s_b P2 + s_a s_b P3 with
// P1 = sum X / 2, P2 = sum Y / 2, P3 = (A/2)(sum sy X + sum sx Y), s_0 = -1, s_1 = 1.
// ---------------------------------------------------------------------------
template <typename T>
__host__ __device__ __forceinline__ T rsqrt_t(T x);
template <>
__host__ __device__ __forceinline__ double rsqrt_t<double>(double x) { return 1.0 / sqrt(x); }
template <>
__host__ __device__ __forceinline__ float rsqrt_t<float>(float x) { return 1.0f / sqrtf(x); }

template <typename T>
__host__ __device__ __forceinline__ void elem_minsurf2(const T u[4], T inv_h2, T r[4]) {
    const T HA = T(0.28867513459481288225);  // A/2 = 1/(2 sqrt 3)
    T p0 = u[0] + u[1], q0 = u[1] - u[0];
    T p1 = u[2] + u[3], q1 = u[3] - u[2];
    T M10 = q0 + q1, M01 = p1 - p0, M11 = q1 - q0;
    const T gx0 = T(0.5) * M10, gy0 = T(0.5) * M01, gd = HA * M11;
    const T gxm = gx0 - gd, gxp = gx0 + gd;  // Gx(sy = -1), Gx(sy = +1)
    const T gym = gy0 - gd, gyp = gy0 + gd;  // Gy(sx = -1), Gy(sx = +1)
    const T axm = gxm * gxm, axp = gxp * gxp, aym = gym * gym, ayp = gyp * gyp;
    // c at (sx, sy)
    const T cmm = rsqrt_t<T>(T(1) + (axm + aym) * inv_h2);
    const T cpm = rsqrt_t<T>(T(1) + (axm + ayp) * inv_h2);
    const T cmp = rsqrt_t<T>(T(1) + (axp + aym) * inv_h2);
    const T cpp = rsqrt_t<T>(T(1) + (axp + ayp) * inv_h2);
    // sums over sx of c at fixed sy (x flux) and over sy at fixed sx (y flux), times 1/4
    const T Xm = T(0.25) * gxm * (cmm + cpm), Xp = T(0.25) * gxp * (cmp + cpp);
    const T Ym = T(0.25) * gym * (cmm + cmp), Yp = T(0.25) * gyp * (cpm + cpp);
    const T P1 = T(0.5) * (Xm + Xp);
    const T P2 = T(0.5) * (Ym + Yp);
    const T P3 = HA * ((Xp - Xm) + (Yp - Ym));
    r[0] = P3 - P1 - P2;
    r[1] = P1 - P2 - P3;
    r[2] = P2 - P1 - P3;
    r[3] = P1 + P2 + P3;
}

// ---------------------------------------------------------------------------
// Neo-Hookean hexahedron of the hyperelastic beam (Sec. 3, "Hyperelasticity").
//   u[3c + i]: displacement component i at corner c = dx + 2 dy + 4 dz
//   inv_h:     1 / h (cube of side h)
//   r[3c + i]: int_e P(F) grad phi_c, component i, with the 2x2x2 Gauss rule,
//              F = I + grad u, J = det F, P = mu F + (lam ln J - mu) F^-T
//              (the stress of W = mu/2 (I_C - 3) - mu ln J + lam/2 (ln J)^2);
//              F^-T = cof(F) / J.  J <= 0 gives a non-finite residual.
// E = 10, nu = 0.3 (Sec. 3): mu = E / (2 (1 + nu)), lam = E nu / ((1 + nu)(1 - 2 nu)).
// Direct evaluation: the beam grids are small, so no factorisation is used.
// ---------------------------------------------------------------------------
constexpr double kBeamMu = 10.0 / (2.0 * 1.3);
constexpr double kBeamLambda = 10.0 * 0.3 / (1.3 * 0.4);

template <typename T>
__host__ __device__ __forceinline__ T log_t(T x);
template <>
__host__ __device__ __forceinline__ double log_t<double>(double x) { return log(x); }
template <>
__host__ __device__ __forceinline__ float log_t<float>(float x) { return logf(x); }

template <typename T>
__host__ __device__ inline void elem_neohooke(const T u[24], T inv_h, T r[24]) {
    const T A = T(0.28867513459481288225);  // 1/(2 sqrt 3)
    const T mu = T(kBeamMu), lam = T(kBeamLambda);
    const T h = T(1) / inv_h;
    const T w = T(0.125) * h * h * h;
#pragma unroll
    for (int k = 0; k < 24; ++k) r[k] = T(0);
#pragma unroll 1
    for (int q = 0; q < 8; ++q) {
        const T px = (q & 1) ? T(0.5) + A : T(0.5) - A;
        const T py = (q & 2) ? T(0.5) + A : T(0.5) - A;
        const T pz = (q & 4) ? T(0.5) + A : T(0.5) - A;
        T G[3][3] = {{T(0), T(0), T(0)}, {T(0), T(0), T(0)}, {T(0), T(0), T(0)}};
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const T sx = (c & 1) ? px : T(1) - px, sy = (c & 2) ? py : T(1) - py, sz = (c & 4) ? pz : T(1) - pz;
            const T gx = ((c & 1) ? inv_h : -inv_h) * sy * sz;
            const T gy = ((c & 2) ? inv_h : -inv_h) * sx * sz;
            const T gz = ((c & 4) ? inv_h : -inv_h) * sx * sy;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                G[i][0] += u[3 * c + i] * gx;
                G[i][1] += u[3 * c + i] * gy;
                G[i][2] += u[3 * c + i] * gz;
            }
        }
        const T F00 = T(1) + G[0][0], F01 = G[0][1], F02 = G[0][2];
        const T F10 = G[1][0], F11 = T(1) + G[1][1], F12 = G[1][2];
        const T F20 = G[2][0], F21 = G[2][1], F22 = T(1) + G[2][2];
        const T C00 = F11 * F22 - F12 * F21, C01 = F12 * F20 - F10 * F22, C02 = F10 * F21 - F11 * F20;
        const T C10 = F02 * F21 - F01 * F22, C11 = F00 * F22 - F02 * F20, C12 = F01 * F20 - F00 * F21;
        const T C20 = F01 * F12 - F02 * F11, C21 = F02 * F10 - F00 * F12, C22 = F00 * F11 - F01 * F10;
        const T J = F00 * C00 + F01 * C01 + F02 * C02;
        const T kc = (lam * log_t<T>(J) - mu) / J;
        const T P[3][3] = {{mu * F00 + kc * C00, mu * F01 + kc * C01, mu * F02 + kc * C02},
                           {mu * F10 + kc * C10, mu * F11 + kc * C11, mu * F12 + kc * C12},
                           {mu * F20 + kc * C20, mu * F21 + kc * C21, mu * F22 + kc * C22}};
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const T sx = (c & 1) ? px : T(1) - px, sy = (c & 2) ? py : T(1) - py, sz = (c & 4) ? pz : T(1) - pz;
            const T gx = ((c & 1) ? inv_h : -inv_h) * sy * sz;
            const T gy = ((c & 2) ? inv_h : -inv_h) * sx * sz;
            const T gz = ((c & 4) ? inv_h : -inv_h) * sx * sy;
#pragma unroll
            for (int i = 0; i < 3; ++i) r[3 * c + i] += w * (P[i][0] * gx + P[i][1] * gy + P[i][2] * gz);
        }
    }
}

}  // namespace jfnk
