// far_math.cuh -- the far-pair Galerkin quadrature of the PMCHWT blocks (paper
// Sec. II-B, Eqs. (K), (T), (Z)) as device functions shared by the far-pair
// kernel (k_assembly.cu) and the fused assembly-projection kernel (k_fused.cu).
// The moment form and the reading of the T sign are described in k_assembly.cu.
#pragma once

#include "internal.cuh"

namespace cbfm {
namespace fm {

constexpr int NCOMP = 27;   // 3 operators x 3 x 3
// Algorithmic work of one quadrature point pair, both media, counting an FMA
// as 2: the direct evaluation of G and g (distance, R, 1/R, e^{-jkR}, the
// (1 + jkR)/R^2 factor) and of the 14 complex moment sums of the far pair
// (sum G, G r, G r', G r.r', g (r x r'), g (r - r')) per medium, about 170
// flops.  The kernel reaches the same sums with fewer operations (moment
// form, shared geometry); the achieved rate is quoted on this count.
constexpr double FAR_FLOP_PER_POINT_PAIR = 170.0;

struct Media {
    double k1r, k1i, k2r, k2i;
    double e1r, e1i, e2r, e2i;   // eta1, eta2
    double f1r, f1i, f2r, f2i;   // 4 / k1^2, 4 / k2^2
    double i1r, i1i, i2r, i2i;   // 1 / eta1, 1 / eta2
};

// the derived constants of a Media from k1, k2, eta1, eta2 (host)
inline Media media_full(z64 k1, z64 k2, z64 e1, z64 e2) {
    const z64 f1 = cdiv(z64(4.0, 0.0), k1 * k1), f2 = cdiv(z64(4.0, 0.0), k2 * k2);
    const z64 i1 = cdiv(z64(1.0, 0.0), e1), i2 = cdiv(z64(1.0, 0.0), e2);
    return Media{k1.re, k1.im, k2.re, k2.im, e1.re, e1.im, e2.re, e2.im,
                 f1.re, f1.im, f2.re, f2.im, i1.re, i1.im, i2.re, i2.im};
}

// Per-medium constants in the arithmetic type of the far-pair kernel,
// computed once on the host: k, 4/k^2 and the operator weights of T into
// Ta = -(eta1 T1 + eta2 T2) and Tb = T1/eta1 + T2/eta2.
template <typename T>
struct MediaT {
    T kr[2], ki[2];
    T fk2r[2], fk2i[2];          // 4 / k^2
    T wTar[2], wTai[2];          // -eta_i
    T wTbr[2], wTbi[2];          // 1 / eta_i
};

template <typename T>
MediaT<T> media_t(const Media &md) {
    MediaT<T> o;
    const double kr[2] = {md.k1r, md.k2r}, ki[2] = {md.k1i, md.k2i};
    const double er[2] = {md.e1r, md.e2r}, ei[2] = {md.e1i, md.e2i};
    for (int i = 0; i < 2; ++i) {
        o.kr[i] = (T)kr[i];
        o.ki[i] = (T)ki[i];
        z64 kk = z64(kr[i], ki[i]) * z64(kr[i], ki[i]);
        z64 f = cdiv(z64(4.0, 0.0), kk);
        o.fk2r[i] = (T)f.re;
        o.fk2i[i] = (T)f.im;
        o.wTar[i] = (T)-er[i];
        o.wTai[i] = (T)-ei[i];
        z64 ie = cdiv(z64(1.0, 0.0), z64(er[i], ei[i]));
        o.wTbr[i] = (T)ie.re;
        o.wTbi[i] = (T)ie.im;
    }
    return o;
}

__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }
__device__ __forceinline__ float exp_t(float x) { return __expf(x); }
__device__ __forceinline__ double exp_t(double x) { return exp(x); }

template <typename T>
struct Mom {
    cx<T> M0, Mrs, MrX;
    cx<T> Mr[3], Ms[3], MW[3], MrW[3], MX[3];
    cx<T> A0, A1[3], B0[3], B1[3];   // far kernel: sums over the test points that give MW, MX, MrW, MrX
};

template <typename T>
__device__ __forceinline__ void zero(Mom<T> &m) {   // the accumulated sums (MW, MX, MrW, MrX are formed after)
    m.M0 = m.Mrs = m.A0 = cx<T>(0, 0);
    for (int d = 0; d < 3; ++d) m.Mr[d] = m.Ms[d] = m.A1[d] = m.B0[d] = m.B1[d] = cx<T>(0, 0);
}

__device__ __forceinline__ bool shares_vertex(const int32_t *a, const int32_t *b) {
    bool r = false;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) r |= (a[i] == b[j]);
    return r;
}

__device__ __forceinline__ double norm3_rn(double x, double y, double z) {
    return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z)));
}

// identical to the classification used for the near list
__device__ __forceinline__ bool is_near(const double *rt, const double *rs, const int32_t *vt, const int32_t *vs,
                                        double alpha) {
    if (shares_vertex(vt, vs)) return true;
    double dx = __dsub_rn(rt[TR_CEN], rs[TR_CEN]);
    double dy = __dsub_rn(rt[TR_CEN + 1], rs[TR_CEN + 1]);
    double dz = __dsub_rn(rt[TR_CEN + 2], rs[TR_CEN + 2]);
    double h = fmax(rt[TR_H], rs[TR_H]);
    return norm3_rn(dx, dy, dz) < __dmul_rn(alpha, h);
}

// Entries of one medium from its moments; adds into out[27] with the
// operator weights (wK for K into Ks; wTa, wTb for T into Ta, Tb).  The
// brackets are split into parts of the trial vertex b and of the test
// vertex a:
//   T: Mrs - pb.Mr - pa.Ms + (pa.pb - 4/k^2) M0 = u_b - v_a + (pa.pb) M0,
//      u_b = Mrs - pb.Mr - (4/k^2) M0,  v_a = pa.Ms
//   K: MrX - pa.MX - pb.MrW + pa.(MW x pb) = y_b + pa.z_b,
//      y_b = MrX - pb.MrW,  z_b = MW x pb - MX
// papb[a][b] = pa.pb and cc[a][b] = c_a c_b are shared by the two media.
template <typename T>
__device__ __forceinline__ void fold_entries(const Mom<T> &m, T kr, T ki, cx<T> four_k2, const T cc[3][3],
                                             const T papb[3][3], const T pa[3][3], const T pb[3][3], cx<T> wTa,
                                             cx<T> wTb, cx<T> *out) {
    const cx<T> mjk(ki, -kr);   // -j k for complex k
    const cx<T> k2M0 = four_k2 * m.M0;
    cx<T> u[3], y[3], z[3][3], v[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        u[b] = m.Mrs - k2M0;
        y[b] = m.MrX;
        for (int d = 0; d < 3; ++d) {
            u[b] -= pb[b][d] * m.Mr[d];
            y[b] -= pb[b][d] * m.MrW[d];
        }
        z[b][0] = m.MW[1] * pb[b][2] - m.MW[2] * pb[b][1] - m.MX[0];
        z[b][1] = m.MW[2] * pb[b][0] - m.MW[0] * pb[b][2] - m.MX[1];
        z[b][2] = m.MW[0] * pb[b][1] - m.MW[1] * pb[b][0] - m.MX[2];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) v[a] = pa[a][0] * m.Ms[0] + pa[a][1] * m.Ms[1] + pa[a][2] * m.Ms[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const cx<T> tb = u[b] - v[a] + papb[a][b] * m.M0;
            const cx<T> kb = y[b] + pa[a][0] * z[b][0] + pa[a][1] * z[b][1] + pa[a][2] * z[b][2];
            const cx<T> Tab = (cc[a][b] * mjk) * tb;
            out[0 * 9 + 3 * a + b] += cc[a][b] * kb;
            out[1 * 9 + 3 * a + b] += wTa * Tab;
            out[2 * 9 + 3 * a + b] += wTb * Tab;
        }
    }
}

// Near test for the far kernel: the squared centroid distance in the kernel's
// type decides all pairs clear of the threshold by a relative margin of 1e-5;
// only pairs inside that band repeat the exact FP64 test of the near list.
template <typename T>
__device__ __forceinline__ bool is_near_t(const T *rt_cen, const T *rt_lo, T ht, const T *rs, const double *rt64,
                                          const double *rs64, const int32_t *vt, const int32_t *vs, double alpha) {
    if (shares_vertex(vt, vs)) return true;
    T d2 = 0;
    for (int d = 0; d < 3; ++d) {
        T dd = (rt_cen[d] - rs[TR_CEN + d]);
        if constexpr (sizeof(T) == 4) dd += (rt_lo[d] - rs[TR_CLO + d]);
        d2 += dd * dd;
    }
    T h = ht > rs[TR_H] ? ht : rs[TR_H];
    T thr = (T)alpha * h;
    T thr2 = thr * thr;
    if (d2 < thr2 * (T)(1.0 - 1e-5)) return true;
    if (d2 > thr2 * (T)(1.0 + 1e-5)) return false;
    return is_near(rt64, rs64, vt, vs, alpha);
}

// The 27 local entries (op x 3 x 3, op = Ks, Ta, Tb) of a far triangle pair:
// rt is the record of the test triangle, rs that of the trial triangle (the
// kernel's type; FP32 records carry the centroid as hi + lo).
// SOA: the test record is stored field-major, element f at rt[f * rts] (a
// structure-of-arrays copy whose consecutive triangles sit in consecutive
// lanes); otherwise at rt[f].
template <typename T, bool SOA = false>
__device__ __forceinline__ void far_entries(const T *rt, int64_t rts, const T *rs, const MediaT<T> &md, cx<T> *out) {
    auto R = [&](int f) -> T { return SOA ? rt[(int64_t)f * rts] : rt[f]; };
    auto sq = [&](int i) -> T { return R(TR_Q + i); };
    auto sw = [&](int i) -> T { return R(TR_W + i); };
    auto sp = [&](int i) -> T { return R(TR_P + i); };
    auto sc = [&](int i) -> T { return R(TR_C + i); };
    auto scen = [&](int i) -> T { return R(TR_CEN + i); };
    auto sclo = [&](int i) -> T { return R(TR_CLO + i); };
    // trial data (local to its centroid)
    T cs[3] = {rs[TR_CEN], rs[TR_CEN + 1], rs[TR_CEN + 2]};
    T ct[3] = {scen(0), scen(1), scen(2)};
    // centroid difference: hi/lo parts in the FP32 records keep it FP64-accurate
    T dc[3];
    for (int d = 0; d < 3; ++d) {
        dc[d] = ct[d] - cs[d];
        if constexpr (sizeof(T) == 4) dc[d] += sclo(d) - rs[TR_CLO + d];
    }
    T rq[7][3], wq[7];
    const T inv4pi = (T)(1.0 / (4.0 * PI));
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        for (int d = 0; d < 3; ++d) rq[q][d] = rs[TR_Q + 3 * q + d] - cs[d];
        wq[q] = rs[TR_W + q] * inv4pi;
    }
    const T kr[2] = {md.kr[0], md.kr[1]};
    const T ki[2] = {md.ki[0], md.ki[1]};
    const bool lossy2 = md.ki[1] != (T)0;
    Mom<T> mm[2];
    zero(mm[0]);
    zero(mm[1]);
    for (int p = 0; p < 7; ++p) {
        T rho[3] = {sq(3 * p) - ct[0], sq(3 * p + 1) - ct[1], sq(3 * p + 2) - ct[2]};
        T Dp[3] = {dc[0] + rho[0], dc[1] + rho[1], dc[2] + rho[2]};
        // per medium over the trial points: S0 = sum w G, S1 = sum w G rho',
        // Sg = sum w g, Y = sum w g rho'.  With d = Dp - rho' (and rho' x rho' = 0)
        // the sums of the definition follow per test point:
        //   W = sum w g d = Dp Sg - Y,  X = sum w g (d x rho') = Dp x Y.
        cx<T> S0[2], S1[2][3], Sg[2], Y[2][3];
        for (int i = 0; i < 2; ++i) {
            S0[i] = Sg[i] = cx<T>(0, 0);
            for (int d = 0; d < 3; ++d) S1[i][d] = Y[i][d] = cx<T>(0, 0);
        }
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            const T d0 = Dp[0] - rq[q][0], d1 = Dp[1] - rq[q][1], d2 = Dp[2] - rq[q][2];
            const T R2 = d0 * d0 + d1 * d1 + d2 * d2;
            const T iR = rsqrt_t(R2);
            const T R = R2 * iR;
            const T niR2 = -(iR * iR);
            const T amp = iR * wq[q];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const T kR = kr[i] * R;
                T sn, cs_;
                sincos_red(kR, &sn, &cs_);
                T a_i = amp;
                if (i == 1 && lossy2) a_i *= exp_t(ki[i] * R);
                // w G = amp (cos - j sin);  w g = -(1 + j k R) w G / R^2, j k R = -ki R + j kr R
                const cx<T> wG(a_i * cs_, -a_i * sn);
                T gx, gy;
                if (i == 1 && lossy2) {
                    const T o = (T)1 - ki[i] * R;
                    gx = o * wG.re - kR * wG.im;
                    gy = o * wG.im + kR * wG.re;
                } else {
                    gx = wG.re - kR * wG.im;
                    gy = wG.im + kR * wG.re;
                }
                const cx<T> wg(niR2 * gx, niR2 * gy);
                S0[i] += wG;
                Sg[i] += wg;
                for (int d = 0; d < 3; ++d) {
                    S1[i][d] += rq[q][d] * wG;
                    Y[i][d] += rq[q][d] * wg;
                }
            }
        }
        const T wp = sw(p);
        const T rw[3] = {wp * rho[0], wp * rho[1], wp * rho[2]};
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            Mom<T> &m = mm[i];
            m.M0 += wp * S0[i];
            m.A0 += wp * Sg[i];
            for (int d = 0; d < 3; ++d) {
                m.Mr[d] += rw[d] * S0[i];
                m.Ms[d] += wp * S1[i][d];
                m.Mrs += rw[d] * S1[i][d];
                m.A1[d] += rw[d] * Sg[i];
                m.B0[d] += wp * Y[i][d];
            }
            // B1 += w rho x Y
            m.B1[0] += rw[1] * Y[i][2] - rw[2] * Y[i][1];
            m.B1[1] += rw[2] * Y[i][0] - rw[0] * Y[i][2];
            m.B1[2] += rw[0] * Y[i][1] - rw[1] * Y[i][0];
        }
    }
    // K moments from the sums over the test points (Dp = dc + rho):
    //   MW = dc A0 + A1 - B0,  MX = dc x B0 + B1,  MrW = A1 x dc - B1,  MrX = -dc.B1
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        Mom<T> &m = mm[i];
        cx<T> MW[3], MX[3], MrW[3];
        for (int d = 0; d < 3; ++d) MW[d] = dc[d] * m.A0 + m.A1[d] - m.B0[d];
        MX[0] = dc[1] * m.B0[2] - dc[2] * m.B0[1] + m.B1[0];
        MX[1] = dc[2] * m.B0[0] - dc[0] * m.B0[2] + m.B1[1];
        MX[2] = dc[0] * m.B0[1] - dc[1] * m.B0[0] + m.B1[2];
        MrW[0] = m.A1[1] * dc[2] - m.A1[2] * dc[1] - m.B1[0];
        MrW[1] = m.A1[2] * dc[0] - m.A1[0] * dc[2] - m.B1[1];
        MrW[2] = m.A1[0] * dc[1] - m.A1[1] * dc[0] - m.B1[2];
        m.MrX = -(dc[0] * m.B1[0] + dc[1] * m.B1[1] + dc[2] * m.B1[2]);
        for (int d = 0; d < 3; ++d) {
            m.MW[d] = MW[d];
            m.MX[d] = MX[d];
            m.MrW[d] = MrW[d];
        }
    }
    // local vertex offsets and coefficients
    T pa[3][3], pb[3][3], cc[3][3], papb[3][3];
    for (int a = 0; a < 3; ++a) {
        for (int d = 0; d < 3; ++d) {
            pa[a][d] = sp(3 * a + d) - ct[d];
            pb[a][d] = rs[TR_P + 3 * a + d] - cs[d];
        }
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            cc[a][b] = sc(a) * rs[TR_C + b];
            papb[a][b] = pa[a][0] * pb[b][0] + pa[a][1] * pb[b][1] + pa[a][2] * pb[b][2];
        }
    // Ks = K1 + K2, Ta = -(eta1 T1 + eta2 T2), Tb = T1/eta1 + T2/eta2
    for (int c = 0; c < NCOMP; ++c) out[c] = cx<T>(0, 0);
#pragma unroll
    for (int i = 0; i < 2; ++i)
        fold_entries<T>(mm[i], kr[i], ki[i], cx<T>(md.fk2r[i], md.fk2i[i]), cc, papb, pa, pb,
                        cx<T>(md.wTar[i], md.wTai[i]), cx<T>(md.wTbr[i], md.wTbi[i]), out);
}


}  // namespace fm
}  // namespace cbfm
