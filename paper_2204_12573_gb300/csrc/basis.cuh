// Radial basis, cutoff and real spherical harmonics (l <= 3) in FP32.
//
// phi_{n,l,m}(r) = T_n(2|r|/r_cut - 1) (r_cut - |r|)^2 Y_lm(r/|r|)   (Sec. V-B:
// radial functions times spherical harmonics, summed into A).  The harmonics
// are real and orthonormal on the sphere; each is written as a homogeneous
// polynomial P_lm of degree l evaluated at the unit vector u, so that
// grad_r Y_lm(r/|r|) = (grad P_lm(u) - l Y_lm(u) u) / |r|.
#pragma once

namespace flr {

// normalisation constants of the real harmonics
constexpr float kY00 = 0.28209479177387814f;   // (1/2) sqrt(1/pi)
constexpr float kY1 = 0.4886025119029199f;     // sqrt(3/(4 pi))
constexpr float kY2a = 1.0925484305920792f;    // (1/2) sqrt(15/pi)
constexpr float kY20 = 0.31539156525252005f;   // (1/4) sqrt(5/pi)
constexpr float kY22 = 0.5462742152960396f;    // (1/4) sqrt(15/pi)
constexpr float kY33 = 0.5900435899266435f;    // (1/4) sqrt(35/(2 pi))
constexpr float kY32 = 2.890611442640554f;     // (1/2) sqrt(105/pi)
constexpr float kY31 = 0.4570457994644658f;    // (1/4) sqrt(21/(2 pi))
constexpr float kY30 = 0.3731763325901154f;    // (1/4) sqrt(7/pi)
constexpr float kY32b = 1.445305721320277f;    // (1/4) sqrt(105/pi)

// Y[l*l + m + l] of a unit vector (x, y, z)
__device__ __forceinline__ void real_ylm(float x, float y, float z, float Y[16])
{
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[0] = kY00;
    Y[1] = kY1 * y;
    Y[2] = kY1 * z;
    Y[3] = kY1 * x;
    Y[4] = kY2a * x * y;
    Y[5] = kY2a * y * z;
    Y[6] = kY20 * (2.f * zz - xx - yy);
    Y[7] = kY2a * x * z;
    Y[8] = kY22 * (xx - yy);
    Y[9] = kY33 * y * (3.f * xx - yy);
    Y[10] = kY32 * x * y * z;
    Y[11] = kY31 * y * (4.f * zz - xx - yy);
    Y[12] = kY30 * z * (2.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = kY31 * x * (4.f * zz - xx - yy);
    Y[14] = kY32b * z * (xx - yy);
    Y[15] = kY33 * x * (xx - 3.f * yy);
}

// sum_lm c[lm] grad P_lm(u) and sum_lm l c[lm] Y_lm(u) (P_lm homogeneous of degree l)
__device__ __forceinline__ void ylm_grad_contract(float x, float y, float z, const float c[16],
                                                  const float Y[16], float &gx, float &gy, float &gz,
                                                  float &lsum)
{
    const float xx = x * x, yy = y * y, zz = z * z;
    gx = 0.f;
    gy = 0.f;
    gz = 0.f;
    // l = 1
    gy += kY1 * c[1];
    gz += kY1 * c[2];
    gx += kY1 * c[3];
    // l = 2
    gx += kY2a * (c[4] * y + c[7] * z) + kY20 * c[6] * (-2.f * x) + kY22 * c[8] * (2.f * x);
    gy += kY2a * (c[4] * x + c[5] * z) + kY20 * c[6] * (-2.f * y) + kY22 * c[8] * (-2.f * y);
    gz += kY2a * (c[5] * y + c[7] * x) + kY20 * c[6] * (4.f * z);
    // l = 3
    gx += kY33 * c[9] * (6.f * x * y) + kY32 * c[10] * (y * z) + kY31 * c[11] * (-2.f * x * y) +
          kY30 * c[12] * (-6.f * x * z) + kY31 * c[13] * (4.f * zz - 3.f * xx - yy) +
          kY32b * c[14] * (2.f * x * z) + kY33 * c[15] * (3.f * xx - 3.f * yy);
    gy += kY33 * c[9] * (3.f * xx - 3.f * yy) + kY32 * c[10] * (x * z) +
          kY31 * c[11] * (4.f * zz - xx - 3.f * yy) + kY30 * c[12] * (-6.f * y * z) +
          kY31 * c[13] * (-2.f * x * y) + kY32b * c[14] * (-2.f * y * z) + kY33 * c[15] * (-6.f * x * y);
    gz += kY32 * c[10] * (x * y) + kY31 * c[11] * (8.f * y * z) +
          kY30 * c[12] * (6.f * zz - 3.f * xx - 3.f * yy) + kY31 * c[13] * (8.f * x * z) +
          kY32b * c[14] * (xx - yy);
    lsum = (c[1] * Y[1] + c[2] * Y[2] + c[3] * Y[3]) +
           2.f * (c[4] * Y[4] + c[5] * Y[5] + c[6] * Y[6] + c[7] * Y[7] + c[8] * Y[8]) +
           3.f * (c[9] * Y[9] + c[10] * Y[10] + c[11] * Y[11] + c[12] * Y[12] + c[13] * Y[13] +
                  c[14] * Y[14] + c[15] * Y[15]);
}

// One harmonic: Y_lm(u) and grad P_lm(u) for a compile-time lm (after
// unrolling, the switch folds away).
__device__ __forceinline__ void ylm_one(int lm, float x, float y, float z, float xx, float yy, float zz,
                                        float &Y, float &dx, float &dy, float &dz)
{
    switch (lm) {
    case 0: Y = kY00; dx = 0.f; dy = 0.f; dz = 0.f; break;
    case 1: Y = kY1 * y; dx = 0.f; dy = kY1; dz = 0.f; break;
    case 2: Y = kY1 * z; dx = 0.f; dy = 0.f; dz = kY1; break;
    case 3: Y = kY1 * x; dx = kY1; dy = 0.f; dz = 0.f; break;
    case 4: Y = kY2a * x * y; dx = kY2a * y; dy = kY2a * x; dz = 0.f; break;
    case 5: Y = kY2a * y * z; dx = 0.f; dy = kY2a * z; dz = kY2a * y; break;
    case 6: Y = kY20 * (2.f * zz - xx - yy); dx = -2.f * kY20 * x; dy = -2.f * kY20 * y; dz = 4.f * kY20 * z; break;
    case 7: Y = kY2a * x * z; dx = kY2a * z; dy = 0.f; dz = kY2a * x; break;
    case 8: Y = kY22 * (xx - yy); dx = 2.f * kY22 * x; dy = -2.f * kY22 * y; dz = 0.f; break;
    case 9: Y = kY33 * y * (3.f * xx - yy); dx = 6.f * kY33 * x * y; dy = kY33 * (3.f * xx - 3.f * yy); dz = 0.f; break;
    case 10: Y = kY32 * x * y * z; dx = kY32 * y * z; dy = kY32 * x * z; dz = kY32 * x * y; break;
    case 11:
        Y = kY31 * y * (4.f * zz - xx - yy);
        dx = -2.f * kY31 * x * y; dy = kY31 * (4.f * zz - xx - 3.f * yy); dz = 8.f * kY31 * y * z;
        break;
    case 12:
        Y = kY30 * z * (2.f * zz - 3.f * xx - 3.f * yy);
        dx = -6.f * kY30 * x * z; dy = -6.f * kY30 * y * z; dz = kY30 * (6.f * zz - 3.f * xx - 3.f * yy);
        break;
    case 13:
        Y = kY31 * x * (4.f * zz - xx - yy);
        dx = kY31 * (4.f * zz - 3.f * xx - yy); dy = -2.f * kY31 * x * y; dz = 8.f * kY31 * x * z;
        break;
    case 14: Y = kY32b * z * (xx - yy); dx = 2.f * kY32b * x * z; dy = -2.f * kY32b * y * z; dz = kY32b * (xx - yy); break;
    default: Y = kY33 * x * (xx - 3.f * yy); dx = kY33 * (3.f * xx - 3.f * yy); dy = -6.f * kY33 * x * y; dz = 0.f; break;
    }
}

// Whether component c (x, y, z) of grad P_lm is not identically zero (lm and
// c compile-time constants after unrolling, so the test folds away).
__host__ __device__ constexpr bool grad_nz(int lm, int c)
{
    // bit lm of each mask: x: 3,4,6-15; y: 1,4,5,6,8-15; z: 2,5,6,7,10-14
    return ((c == 0 ? 0xFFD8u : (c == 1 ? 0xFF72u : 0x7CE4u)) >> lm) & 1u;
}

// l of harmonic index lm
__host__ __device__ constexpr int l_of(int lm) { return lm < 1 ? 0 : (lm < 4 ? 1 : (lm < 9 ? 2 : 3)); }

// T_n(x) (r_cut - r)^2 for n < N, and optionally its r-derivative;
// tr = 2 / r_cut, so x = r tr - 1 needs no division per pair
template <int N, bool GRAD>
__device__ __forceinline__ void radial(float r, float rc, float tr, float Rf[N], float dRf[N])
{
    const float x = r * tr - 1.f;
    const float dxdr = tr;
    const float t = rc - r;
    const float fc = t * t;
    const float dfc = -2.f * t;
    float tm2 = 1.f, tm1 = x;        // T_0, T_1
    float dm2 = 0.f, dm1 = 1.f;      // T_0', T_1' (d/dx)
#pragma unroll
    for (int n = 0; n < N; ++n) {
        float T, dT;
        if (n == 0) {
            T = 1.f;
            dT = 0.f;
        } else if (n == 1) {
            T = x;
            dT = 1.f;
        } else {
            T = 2.f * x * tm1 - tm2;
            dT = 2.f * tm1 + 2.f * x * dm1 - dm2;
            tm2 = tm1;
            tm1 = T;
            dm2 = dm1;
            dm1 = dT;
        }
        Rf[n] = T * fc;
        if (GRAD) dRf[n] = dT * dxdr * fc + T * dfc;
    }
}

// T_n(x) and dT_n/dx for 2 <= n < N (T_0 = 1, T_1 = x, T_0' = 0, T_1' = 1
// are left to the caller, which folds them into its sums)
template <int N>
__device__ __forceinline__ void cheb_tail(float x, float T[N], float dT[N])
{
    float tm2 = 1.f, tm1 = x;
    float dm2 = 0.f, dm1 = 1.f;
#pragma unroll
    for (int n = 2; n < N; ++n) {
        T[n] = 2.f * x * tm1 - tm2;
        dT[n] = 2.f * tm1 + 2.f * x * dm1 - dm2;
        tm2 = tm1;
        tm1 = T[n];
        dm2 = dm1;
        dm1 = dT[n];
    }
}

}  // namespace flr
