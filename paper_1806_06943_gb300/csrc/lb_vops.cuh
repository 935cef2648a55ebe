// lb_vops.cuh -- explicit FP32 arithmetic of the offset-population step,
// written once for a value of one species (float) and of both species
// (Sp<float>).  Every operation is an intrinsic that rounds once, exactly as
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

// a value of each species
template <class T>
struct Sp {
    T a, b;
};
template <class T>
__device__ __forceinline__ Sp<T> vadd(Sp<T> x, Sp<T> y) { return {vadd(x.a, y.a), vadd(x.b, y.b)}; }
template <class T>
__device__ __forceinline__ Sp<T> vsub(Sp<T> x, Sp<T> y) { return {vsub(x.a, y.a), vsub(x.b, y.b)}; }
template <class T>
__device__ __forceinline__ Sp<T> vmul(Sp<T> x, Sp<T> y) { return {vmul(x.a, y.a), vmul(x.b, y.b)}; }
template <class T>
__device__ __forceinline__ Sp<T> vfma(Sp<T> x, Sp<T> y, Sp<T> z) { return {vfma(x.a, y.a, z.a), vfma(x.b, y.b, z.b)}; }
template <class T>
__device__ __forceinline__ Sp<T> vsplat(float c, Sp<T>) { return {vsplat(c, T{}), vsplat(c, T{})}; }

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
// Eq. (3) from the half-force momenta m_k (Eq. 6), -1.5 u.u, -u.F_k, and
// w(|e|^2) rho_k, w(|e|^2) dg_k for the three weight classes (dg_k: the sum
// of the node's offsets from its rounded density).
template <class V>
struct OffTerms {
    V ux, uy, m15uu;
    V nuF[2];
    V F[2][2];
    V wr[2][3], wdg[2][3];
};

template <class V>
__device__ __forceinline__ void off_terms(float om0, float om1, const V (&rho)[2], const V (&m)[2][2], const V (&F)[2][2],
                                          const V (&dg)[2], OffTerms<V> &t)
{
    const V den = cfma(om1, rho[1], cmul(om0, rho[0]));
    const V nx = cfma(om1, m[1][0], cmul(om0, m[0][0]));
    const V ny = cfma(om1, m[1][1], cmul(om0, m[0][1]));
    t.ux = vdiv(nx, den);
    t.uy = vdiv(ny, den);
    t.m15uu = cmul(-1.5f, vfma(t.uy, t.uy, vmul(t.ux, t.ux)));
    const float wc[3] = {(float)(4.0 / 9.0), (float)(1.0 / 9.0), (float)(1.0 / 36.0)};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        t.F[k][0] = F[k][0];
        t.F[k][1] = F[k][1];
        t.nuF[k] = vneg(vfma(t.uy, F[k][1], vmul(t.ux, F[k][0])));
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            t.wr[k][c] = cmul(wc[c], rho[k]);
            t.wdg[k][c] = cmul(wc[c], dg[k]);
        }
    }
}

// Post-collision offset of direction I of species k from its offset f:
// f + omega_k (g^eq - f) + C, with g^eq = w rho_k (3 e.u + 4.5 (e.u)^2 -
// 1.5 u.u) + w dg_k (Eq. 2 less w rho_k) and the Guo term of Eq. (5) as
// C = 3 (1 - omega_k/2) w [(e.F)(1 + 3 e.u) - u.F] (aw3 = 3 (1 - omega_k/2) w),
// added in the fma that forms its last product.
template <int I, class V>
__device__ __forceinline__ V off_collide(const OffTerms<V> &t, int k, float om, float aw3, V f)
{
    constexpr int C = I == 0 ? 0 : (I <= 4 ? 1 : 2);
    V q, X;
    if constexpr (I == 0) {
        q = t.m15uu;
        X = t.nuF[k];
    } else {
        constexpr int B = vbase9(I);
        constexpr float s = vsign9(I);
        const V e = vbase<B>(t.ux, t.uy);                      // e.u = s e
        q = vfma(cmul(4.5f, e), e, cfma(3.f * s, e, t.m15uu));  // 4.5 (e.u)^2 + 3 e.u - 1.5 u.u
        const V tt = cfma(3.f, e, vsplat(s, e));               // s (1 + 3 e.u)
        const V eF = vbase<B>(t.F[k][0], t.F[k][1]);           // e.F = s eF
        X = vfma(eF, tt, t.nuF[k]);
    }
    const V geq = vfma(t.wr[k][C], q, t.wdg[k][C]);
    return cfma(aw3, X, cfma(om, vsub(geq, f), f));
}

}  // namespace lbk
