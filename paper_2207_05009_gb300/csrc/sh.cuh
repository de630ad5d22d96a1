// Real spherical-harmonic basis of the emission (paper Sec. 4.2, Eq. 6) as
// Cartesian polynomials of the unit direction: orthonormal, k = l(l+1)+m,
// m < 0 <-> sin(|m| phi), no Condon-Shortley phase, l <= 3.
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
        }
    }
}

}  // namespace plo
