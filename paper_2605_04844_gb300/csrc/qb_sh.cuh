// qb_sh.cuh -- real spherical-harmonic colour (degree 0..3) and its gradient.
//
// Colour of a Gaussian (Sec. 2, "spherical harmonic coefficients"):
//   rgb = max(0, sum_k sh_k Y_k(d) + 0.5),  d = unit vector campos -> mean.
// Y_k are the real harmonics carrying the Condon-Shortley phase, index
// k = l*l + l + m, written here as homogeneous polynomials in (x, y, z) of
// the unit direction.  The constants are K_l^|m| * sqrt(2)^(m != 0) times the
// Legendre polynomial's leading factor, with
// K_l^m = sqrt((2l+1)/(4 pi) * (l-m)!/(l+m)!):
//   l=0: 1/(2 sqrt(pi))
//   l=1: sqrt(3/(4 pi))
//   l=2: sqrt(15/pi)/2, sqrt(5/pi)/4, sqrt(15/pi)/4
//   l=3: sqrt(35/(2 pi))/4, sqrt(105/pi)/2, sqrt(21/(2 pi))/4, sqrt(7/pi)/4, sqrt(105/pi)/4
#pragma once

namespace qb {

constexpr float kY00 = 0.28209479177387814f;
constexpr float kY1 = 0.48860251190291992f;
constexpr float kY2a = 1.0925484305920792f;   // sqrt(15/pi)/2
constexpr float kY2b = 0.31539156525252005f;  // sqrt(5/pi)/4
constexpr float kY2c = 0.54627421529603959f;  // sqrt(15/pi)/4
constexpr float kY3a = 0.59004358992664352f;  // sqrt(35/(2pi))/4
constexpr float kY3b = 2.8906114426405538f;   // sqrt(105/pi)/2
constexpr float kY3c = 0.45704579946446572f;  // sqrt(21/(2pi))/4
constexpr float kY3d = 0.37317633259011540f;  // sqrt(7/pi)/4
constexpr float kY3e = 1.4453057213202769f;   // sqrt(105/pi)/4

template <int DEG>
__device__ __forceinline__ void sh_eval(float x, float y, float z, float Y[16]) {
    Y[0] = kY00;
    if (DEG >= 1) {
        Y[1] = -kY1 * y;
        Y[2] = kY1 * z;
        Y[3] = -kY1 * x;
    }
    if (DEG >= 2) {
        float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = kY2a * x * y;
        Y[5] = -kY2a * y * z;
        Y[6] = kY2b * (2.f * zz - xx - yy);
        Y[7] = -kY2a * x * z;
        Y[8] = kY2c * (xx - yy);
        if (DEG >= 3) {
            Y[9] = -kY3a * y * (3.f * xx - yy);
            Y[10] = kY3b * x * y * z;
            Y[11] = -kY3c * y * (4.f * zz - xx - yy);
            Y[12] = kY3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = -kY3c * x * (4.f * zz - xx - yy);
            Y[14] = kY3e * z * (xx - yy);
            Y[15] = -kY3a * x * (xx - 3.f * yy);
        }
    }
}

// Gradient of sum_k w_k Y_k(x, y, z) w.r.t. (x, y, z) for the polynomial
// extension of the basis off the sphere (the caller projects out the radial
// component through the normalisation of d).
template <int DEG>
__device__ __forceinline__ void sh_grad(float x, float y, float z, const float w[16], float &gx, float &gy,
                                        float &gz) {
    gx = gy = gz = 0.f;
    if (DEG >= 1) {
        gx += -kY1 * w[3];
        gy += -kY1 * w[1];
        gz += kY1 * w[2];
    }
    if (DEG >= 2) {
        float xx = x * x, yy = y * y, zz = z * z;
        // Y4 = a xy
        gx += kY2a * y * w[4];
        gy += kY2a * x * w[4];
        // Y5 = -a yz
        gy += -kY2a * z * w[5];
        gz += -kY2a * y * w[5];
        // Y6 = b (2zz - xx - yy)
        gx += kY2b * (-2.f * x) * w[6];
        gy += kY2b * (-2.f * y) * w[6];
        gz += kY2b * (4.f * z) * w[6];
        // Y7 = -a xz
        gx += -kY2a * z * w[7];
        gz += -kY2a * x * w[7];
        // Y8 = c (xx - yy)
        gx += kY2c * 2.f * x * w[8];
        gy += kY2c * (-2.f * y) * w[8];
        if (DEG >= 3) {
            // Y9 = -a3 (3xxy - yyy)
            gx += -kY3a * 6.f * x * y * w[9];
            gy += -kY3a * (3.f * xx - 3.f * yy) * w[9];
            // Y10 = b3 xyz
            gx += kY3b * y * z * w[10];
            gy += kY3b * x * z * w[10];
            gz += kY3b * x * y * w[10];
            // Y11 = -c3 (4yzz - xxy - yyy)
            gx += -kY3c * (-2.f * x * y) * w[11];
            gy += -kY3c * (4.f * zz - xx - 3.f * yy) * w[11];
            gz += -kY3c * (8.f * y * z) * w[11];
            // Y12 = d3 (2zzz - 3xxz - 3yyz)
            gx += kY3d * (-6.f * x * z) * w[12];
            gy += kY3d * (-6.f * y * z) * w[12];
            gz += kY3d * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
            // Y13 = -c3 (4xzz - xxx - xyy)
            gx += -kY3c * (4.f * zz - 3.f * xx - yy) * w[13];
            gy += -kY3c * (-2.f * x * y) * w[13];
            gz += -kY3c * (8.f * x * z) * w[13];
            // Y14 = e3 (xxz - yyz)
            gx += kY3e * 2.f * x * z * w[14];
            gy += kY3e * (-2.f * y * z) * w[14];
            gz += kY3e * (xx - yy) * w[14];
            // Y15 = -a3 (xxx - 3xyy)
            gx += -kY3a * (3.f * xx - 3.f * yy) * w[15];
            gy += -kY3a * (-6.f * x * y) * w[15];
        }
    }
}

}  // namespace qb
