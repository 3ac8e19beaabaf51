// rod_update.cuh -- one entry of the frame update of Eq. (newD), shared by the warp-cooperative
// update kernel (rod_kernels.cu) and the update epilogue of the cluster pair-sum kernel
// (mrs_kernels.cu).
//
// Rotating the directors of a node by |w| h about w / |w| (Rodrigues' formula written without
// normalising w; theta^2 = |w|^2 h^2):
//   d_i' = cos(theta) d_i + (sin(theta)/theta) h (w x d_i) + ((1 - cos(theta))/theta^2) h^2 (w.d_i) w,
// the two ratios from their Taylor series in theta^2 when theta^2 < 1e-3 (the next terms are
// below 1e-22: exact in float64) and from sincos otherwise; w = 0 leaves the frame unchanged.
#pragma once

namespace mrs {

// The formula's three coefficients for w and h: d_i' = ct d_i + a (w x d_i) + b (w.d_i) w.
// Returns false (and leaves them unset) when w = 0.
__device__ __forceinline__ bool rodrigues_coefficients(double wx, double wy, double wz, double h,
                                                       double& ct, double& a, double& b)
{
    const double w2 = wx * wx + wy * wy + wz * wz;
    if (w2 == 0.0) return false;
    const double q = w2 * h * h;   // theta^2
    double sc, cc;                 // sin(theta)/theta, (1 - cos(theta))/theta^2
    if (q < 1e-3) {
        sc = 1.0 + q * (-1.0 / 6.0 + q * (1.0 / 120.0 + q * (-1.0 / 5040.0 + q * (1.0 / 362880.0))));
        cc = 0.5 + q * (-1.0 / 24.0 + q * (1.0 / 720.0 + q * (-1.0 / 40320.0 + q * (1.0 / 3628800.0))));
        ct = 1.0 - q * cc;
    } else {
        const double th = sqrt(q);
        double st;
        sincos(th, &st, &ct);
        sc = st / th;
        cc = (1.0 - ct) / q;
    }
    a = sc * h;
    b = cc * h * h;
    return true;
}

// Component c of the new director i, from the old director i = (v0, v1, v2).
__device__ __forceinline__ double rodrigues_entry(double v0, double v1, double v2, double wx, double wy,
                                                  double wz, double h, int c)
{
    const double vc = c == 0 ? v0 : c == 1 ? v1 : v2;
    double ct, a, b;
    if (!rodrigues_coefficients(wx, wy, wz, h, ct, a, b)) return vc;
    const double wv = b * (wx * v0 + wy * v1 + wz * v2);
    // component c of w x d_i = wA vB - wB vA: (wy v2 - wz v1, wz v0 - wx v2, wx v1 - wy v0)
    const double wA = c == 0 ? wy : c == 1 ? wz : wx, vB = c == 0 ? v2 : c == 1 ? v0 : v1;
    const double wB = c == 0 ? wz : c == 1 ? wx : wy, vA = c == 0 ? v1 : c == 1 ? v2 : v0;
    const double cr = wA * vB - wB * vA;
    const double wc = c == 0 ? wx : c == 1 ? wy : wz;
    return ct * vc + a * cr + wv * wc;
}

}  // namespace mrs
