// Real spherical-harmonic basis of the emission (paper Sec. 4.2, Eq. 6) as
// Cartesian polynomials of the unit direction: orthonormal, k = l(l+1)+m,
// m < 0 <-> sin(|m| phi), no Condon-Shortley phase, l <= 4.  Degree 4 (Sec.
// 6.2 compares l_max = 2, 3, 4) with c = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!)
// folded into each constant:
//   m = +-4: (3/4) sqrt(35/pi) xy(x^2-y^2), (3/16) sqrt(35/pi) (x^4 - 6x^2y^2 + y^4)
//   m = +-3: (3/4) sqrt(35/(2pi)) z y(3x^2-y^2), z x(x^2-3y^2)
//   m = +-2: (3/4) sqrt(5/pi) xy(7z^2-1), (3/8) sqrt(5/pi) (x^2-y^2)(7z^2-1)
//   m = +-1: (3/4) sqrt(5/(2pi)) z(7z^2-3) y, x
//   m = 0:   (3/16) sqrt(1/pi) (35z^4 - 30z^2 + 3)
#pragma once

namespace plo {

// Written with explicit rounding intrinsics so that every kernel that inlines
// it computes the same bits (the compiler may not contract these into FMAs
// differently per call site).
template <int K>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float* Y) {
    Y[0] = 0.28209479177387814f;
    if (K > 1) {
        Y[1] = __fmul_rn(0.4886025119029199f, y);
        Y[2] = __fmul_rn(0.4886025119029199f, z);
        Y[3] = __fmul_rn(0.4886025119029199f, x);
    }
    if (K > 4) {
        const float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
        const float xy = __fmul_rn(x, y), yz = __fmul_rn(y, z), xz = __fmul_rn(x, z);
        const float xx_yy = __fsub_rn(xx, yy);
        Y[4] = __fmul_rn(1.0925484305920792f, xy);
        Y[5] = __fmul_rn(1.0925484305920792f, yz);
        Y[6] = __fmul_rn(0.31539156525252005f, __fmaf_rn(3.0f, zz, -1.0f));
        Y[7] = __fmul_rn(1.0925484305920792f, xz);
        Y[8] = __fmul_rn(0.5462742152960396f, xx_yy);
        if (K > 9) {
            const float five_zz_1 = __fmaf_rn(5.0f, zz, -1.0f);
            Y[9] = __fmul_rn(__fmul_rn(0.5900435899266435f, y), __fmaf_rn(3.0f, xx, -yy));
            Y[10] = __fmul_rn(__fmul_rn(2.890611442640554f, xy), z);
            Y[11] = __fmul_rn(__fmul_rn(0.4570457994644658f, y), five_zz_1);
            Y[12] = __fmul_rn(__fmul_rn(0.3731763325901154f, z), __fmaf_rn(5.0f, zz, -3.0f));
            Y[13] = __fmul_rn(__fmul_rn(0.4570457994644658f, x), five_zz_1);
            Y[14] = __fmul_rn(__fmul_rn(1.445305721320277f, z), xx_yy);
            Y[15] = __fmul_rn(__fmul_rn(0.5900435899266435f, x), __fmaf_rn(-3.0f, yy, xx));
            if (K > 16) {
                const float seven_zz_1 = __fmaf_rn(7.0f, zz, -1.0f), seven_zz_3 = __fmaf_rn(7.0f, zz, -3.0f);
                const float x3y = __fmaf_rn(3.0f, xx, -yy), xx3 = __fmaf_rn(-3.0f, yy, xx);
                Y[16] = __fmul_rn(__fmul_rn(2.5033429417967046f, xy), xx_yy);
                Y[17] = __fmul_rn(__fmul_rn(1.7701307697799304f, yz), x3y);
                Y[18] = __fmul_rn(__fmul_rn(0.9461746957575601f, xy), seven_zz_1);
                Y[19] = __fmul_rn(__fmul_rn(0.6690465435572892f, yz), seven_zz_3);
                Y[20] = __fmul_rn(0.10578554691520431f,
                                  __fmaf_rn(zz, __fmaf_rn(35.0f, zz, -30.0f), 3.0f));
                Y[21] = __fmul_rn(__fmul_rn(0.6690465435572892f, xz), seven_zz_3);
                Y[22] = __fmul_rn(__fmul_rn(0.47308734787878004f, xx_yy), seven_zz_1);
                Y[23] = __fmul_rn(__fmul_rn(1.7701307697799304f, xz), xx3);
                Y[24] = __fmul_rn(0.6258357354491761f, __fsub_rn(__fmul_rn(xx, xx3), __fmul_rn(yy, x3y)));
            }
        }
    }
}

}  // namespace plo
