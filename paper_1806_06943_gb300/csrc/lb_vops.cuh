// lb_vops.cuh -- explicit FP32 arithmetic of the offset-population step,
// written once for a value of one species (float) and of both species (a
// float2 pair in the paired FP32 instructions).  Every operation is an
// intrinsic that rounds once, exactly as
// written, and that the compiler never contracts with another, so every FP32
// kernel (two-pass, one-pass, persistent, TMA) evaluates Eqs. (1)-(3), (5),
// (6), (8), (9) with the same roundings, whatever it stages in shared memory
// and however the compiler schedules it.
#pragma once

#include <cuda_runtime.h>

namespace lbk {

__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float vsplat(float c, float) { return c; }
__device__ __forceinline__ float vdiv(float a, float b) { return __fdiv_rn(a, b); }

// A value of each species as one (A, B) pair in Blackwell's paired FP32
// instructions: each lane rounds once, exactly as the scalar intrinsic above,
// so a step written on pairs gives the same bits as one written per species.
// The code generator merges a paired multiply into a paired add that consumes
// it (one FFMA2, whatever the rounding suffix), so nothing here adds a rounded
// product: such sums are written as one fma.  a - b is b * (-1) + a, exact
// before its one rounding.
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vsplat(float c, float2) { return make_float2(c, c); }
// each lane gets the other species' value
__device__ __forceinline__ float2 vswap(float2 a) { return make_float2(a.y, a.x); }

// a constant times / plus a value
template <class V>
__device__ __forceinline__ V cmul(float c, V x) { return vmul(vsplat(c, x), x); }
template <class V>
__device__ __forceinline__ V cfma(float c, V x, V y) { return vfma(vsplat(c, x), x, y); }

// ---- sums of the FP32 step ---------------------------------------------------

// sum_i h_i of one species: the rest population, then the axis and diagonal
// pairs of opposite directions (D2Q9 order rest, (1,0), (0,1), (-1,0),
// (0,-1), (1,1), (-1,1), (-1,-1), (1,-1)).
template <class V>
__device__ __forceinline__ V vzeroth(const V (&f)[9])
{
    return vadd(f[0], vadd(vadd(vadd(f[1], f[3]), vadd(f[2], f[4])), vadd(vadd(f[5], f[7]), vadd(f[6], f[8]))));
}

// sum_i h_i e_i of one species from opposite-population differences
// (exactly antisymmetric under reflection).
template <class V>
__device__ __forceinline__ void vfirst(const V (&f)[9], V &jx, V &jy)
{
    const V d57 = vsub(f[5], f[7]), d86 = vsub(f[8], f[6]);
    jx = vadd(vsub(f[1], f[3]), vadd(d57, d86));
    jy = vadd(vsub(f[2], f[4]), vsub(d57, d86));
}

// sum_{i=1..8} w_i s(x + e_i) e_i (Eqs. 8, 9) from the differences of
// opposite neighbours; at(dy, dx) is the staged value at offset (dx, dy).
template <class V, class At>
__device__ __forceinline__ void vq9(const At &at, V &sx, V &sy)
{
    const float W1 = (float)(1.0 / 9.0), W2 = (float)(1.0 / 36.0);
    const V dE = vsub(at(0, 1), at(0, -1));
    const V dN = vsub(at(1, 0), at(-1, 0));
    const V d1 = vsub(at(1, 1), at(-1, -1));   // (1,1) - (-1,-1)
    const V d2 = vsub(at(-1, 1), at(1, -1));   // (1,-1) - (-1,1)
    sx = cfma(W1, dE, cmul(W2, vadd(d1, d2)));
    sy = cfma(W1, dN, cmul(W2, vsub(d1, d2)));
}

// -sum_j c_j s(x + e_j) e_j over D2Q25 with the weights of the two psi sums
// of Eq. (8) combined, c(|e|^2) = G1 w(|e|^2) + G2 p(|e|^2): the near
// cancellation of the attraction and the repulsion on the inner ring
// (|e|^2 = 1, 2) happens in its two weights, formed in FP64 per lattice,
// instead of between two rounded sums.  cw = (-c(1), -c(2), -G2); the outer
// ring (|e|^2 = 4, 5, 8, where w = 0) is summed with the weights p and then
// scaled by -G2.  Opposite-neighbour differences throughout.
template <class V, class At, class Pf>
__device__ __forceinline__ void vq25c(const At &at, const float (&cw)[3], Pf p25f, V &sx, V &sy)
{
    const V dE = vsub(at(0, 1), at(0, -1));
    const V dN = vsub(at(1, 0), at(-1, 0));
    const V d1 = vsub(at(1, 1), at(-1, -1));   // (1,1) - (-1,-1)
    const V d2 = vsub(at(-1, 1), at(1, -1));   // (1,-1) - (-1,1)
    V ox = cmul(p25f(4) * 2.f, vsub(at(0, 2), at(0, -2)));
    V oy = cmul(p25f(4) * 2.f, vsub(at(2, 0), at(-2, 0)));
#pragma unroll
    for (int a = 1; a <= 2; ++a)
#pragma unroll
        for (int b = 1; b <= 2; ++b) {
            if (a == 1 && b == 1) continue;
            const V e1 = vsub(at(b, a), at(-b, -a));   // (a,b) - (-a,-b)
            const V e2 = vsub(at(-b, a), at(b, -a));   // (a,-b) - (-a,b)
            const float p = p25f(a * a + b * b);
            ox = cfma(p * (float)a, vadd(e1, e2), ox);
            oy = cfma(p * (float)b, vsub(e1, e2), oy);
        }
    sx = cfma(cw[0], dE, cfma(cw[1], vadd(d1, d2), cmul(cw[2], ox)));
    sy = cfma(cw[0], dN, cfma(cw[1], vsub(d1, d2), cmul(cw[2], oy)));
}

// Total force on one species (Eq. 8 + Eq. 9 + rho g) from its combined psi
// sum ms = -sum_j c_j psi(x + e_j) e_j (vq25c) and the other species'
// density sum s3 (vq9): F = psi ms - G_AB rho s3 + rho g.
template <class V>
__device__ __forceinline__ void vforce(V psi, V rho, V msx, V msy, V s3x, V s3y, float GAB, float gx, float gy, V &Fx,
                                       V &Fy)
{
    const V c = cmul(-GAB, rho);
    Fx = vfma(psi, msx, vfma(c, s3x, cmul(gx, rho)));
    Fy = vfma(psi, msy, vfma(c, s3y, cmul(gy, rho)));
}

// ---- the FP32 collision (Eqs. 1-3, 5, 6 on offset populations) ---------------

// D2Q9 direction i as seen by the collision: e_i . v = s * base(v), base 0:
// v_x, 1: v_y, 2: v_x + v_y, 3: v_x - v_y (rest: none).
__host__ __device__ constexpr int vbase9(int i) { return (i == 1 || i == 3) ? 0 : (i == 2 || i == 4) ? 1 : (i == 5 || i == 7) ? 2 : 3; }
__host__ __device__ constexpr float vsign9(int i) { return (i == 3 || i == 4 || i == 7 || i == 6) ? -1.f : 1.f; }

template <int B, class V>
__device__ __forceinline__ V vbase(V x, V y)
{
    if constexpr (B == 0) return x;
    else if constexpr (B == 1) return y;
    else if constexpr (B == 2) return vadd(x, y);
    else return vsub(x, y);
}

template <class V>
__device__ __forceinline__ V vneg(V x) { return vsub(vsplat(0.f, x), x); }

// The node's terms of the collision shared by its directions: u^eq of
// Eq. (3) from the half-force momenta m_k (Eq. 6) and -1.5 u.u, shared by the
// species; per species, as (A, B) pairs, F_k, -u.F_k, and w(|e|^2) rho_k,
// w(|e|^2) dg_k for the three weight classes (dg_k: the sum of the node's
// offsets from its rounded density).
struct OffTerms {
    float ux, uy, m15uu;
    float2 Fx, Fy, nuF;
    float2 wr[3], wdg[3];
};

__device__ __forceinline__ void off_terms(float2 om, float2 rho, float2 mx, float2 my, float2 Fx, float2 Fy, float2 dg,
                                          OffTerms &t)
{
    const float den = vfma(om.y, rho.y, vmul(om.x, rho.x));
    const float nx = vfma(om.y, mx.y, vmul(om.x, mx.x));
    const float ny = vfma(om.y, my.y, vmul(om.x, my.x));
    t.ux = vdiv(nx, den);
    t.uy = vdiv(ny, den);
    t.m15uu = cmul(-1.5f, vfma(t.uy, t.uy, vmul(t.ux, t.ux)));
    t.Fx = Fx;
    t.Fy = Fy;
    t.nuF = vneg(vfma(vsplat(t.uy, Fy), Fy, vmul(vsplat(t.ux, Fx), Fx)));
    const float wc[3] = {(float)(4.0 / 9.0), (float)(1.0 / 9.0), (float)(1.0 / 36.0)};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        t.wr[c] = cmul(wc[c], rho);
        t.wdg[c] = cmul(wc[c], dg);
    }
}

// Post-collision offsets of direction I of both species from their offsets
// f: f + omega_k (g^eq - f) + C, with g^eq = w rho_k (3 e.u + 4.5 (e.u)^2 -
// 1.5 u.u) + w dg_k (Eq. 2 less w rho_k) and the Guo term of Eq. (5) as
// C = 3 (1 - omega_k/2) w [(e.F)(1 + 3 e.u) - u.F] (aw3 = 3 (1 - omega_k/2) w),
// added in the fma that forms its last product.  The terms in e.u are the
// species' common ones.
template <int I>
__device__ __forceinline__ float2 off_collide(const OffTerms &t, float2 om, float2 aw3, float2 f)
{
    constexpr int C = I == 0 ? 0 : (I <= 4 ? 1 : 2);
    float q;
    float2 X;
    if constexpr (I == 0) {
        q = t.m15uu;
        X = t.nuF;
    } else {
        constexpr int B = vbase9(I);
        constexpr float s = vsign9(I);
        const float e = vbase<B>(t.ux, t.uy);                      // e.u = s e
        q = vfma(cmul(4.5f, e), e, cfma(3.f * s, e, t.m15uu));      // 4.5 (e.u)^2 + 3 e.u - 1.5 u.u
        const float tt = cfma(3.f, e, vsplat(s, e));               // s (1 + 3 e.u)
        const float2 eF = vbase<B>(t.Fx, t.Fy);                    // e.F = s eF
        X = vfma(eF, vsplat(tt, eF), t.nuF);
    }
    const float2 geq = vfma(t.wr[C], vsplat(q, f), t.wdg[C]);
    return vfma(aw3, X, vfma(om, vsub(geq, f), f));
}

}  // namespace lbk
