// k_assembly.cu -- Galerkin assembly of the PMCHWT blocks (paper Sec. II-B,
// Eqs. (K), (T), (Z)).
//
// Every stage runs over any number of meshes in one launch (a single mesh is
// a batch of one).
// Stage 1, far pairs (k_far): persistent CTAs take tasks (mesh, test triangle
//   t, strip of trial triangles s >= t) from an atomic counter; one thread per trial
//   triangle s evaluates both media over the 7 x 7 point pairs and reduces them to 18
//   complex moments per medium, from which the 3 x 3 local blocks follow:
//     T_ab = -j k c_a c_b [ Mrs - pi'_b.Mr - pi_a.Ms + (pi_a.pi'_b - 4/k^2) M0 ]
//     K_ab =      c_a c_b [ MrX - pi_a.MX - pi'_b.MrW + pi_a.(MW x pi'_b) ]
//   with positions taken relative to each triangle's centroid (rho on t, rho'
//   on s, pi = vertex - centroid) and d = r - r' = (c_t - c_s) + rho - rho':
//     S0 = sum_q w_q G, S1 = sum_q w_q G rho', W = sum_q w_q g d,
//     X = sum_q w_q g (d x rho'),  G = e^{-jkR}/(4 pi R), g = -(1+jkR) e^{-jkR}/(4 pi R^3)
//     M0 = sum_p w_p S0, Mr = sum_p w_p rho S0, Ms = sum_p w_p S1, Mrs = sum_p w_p rho.S1,
//     MW = sum_p w_p W, MrW = sum_p w_p rho x W, MX = sum_p w_p X, MrX = sum_p w_p rho.X
//   The K sums are evaluated through Sg = sum_q w_q g and Y = sum_q w_q g rho':
//   with Dp = (c_t - c_s) + rho, d x rho' = Dp x rho', so W = Dp Sg - Y and
//   X = Dp x Y, and the sums over p of w_p Sg, w_p rho Sg, w_p Y, w_p rho x Y
//   give MW, MX, MrW, MrX once per pair.
//   The minus sign on T is the reading under which the paper's block matrix
//   describes the exp(+j w t) problem.  Blocks are combined into
//   Ks = K1 + K2, Ta = -(eta1 T1 + eta2 T2), Tb = T1/eta1 + T2/eta2.
// Stage 2, near pairs (k_near_blocks, two pairs per warp; FP64 for the closed
//   forms, and on the mixed path FP32 for the smooth remainders and the outer
//   test-point quadrature): 1/R, 1/R^3 and k^2/(2R)
//   integrated in closed form over the trial triangle (Wilton et al. 1984,
//   Graglia 1993 edge sums), bounded remainders by the 7-point rule, blocks
//   symmetrised L(t,s) = (L~(t,s) + L~(s,t)^T)/2; K of a triangle with itself is 0.
// Stage 3 (k_mirror): the blocks of the pairs s < t, transposed from (s, t).
// Stage 4 (k_gather, one block per RWG row): RWG entries Z_op[i][j] = sum over
//   the 2 x 2 triangle pairs of the two supports.
#include <algorithm>
#include <string>
#include <vector>

#include "far_math.cuh"

namespace cbfm {

namespace {

using namespace fm;

// One staged item of the far kernel, in shared memory: the test triangle t
// (its record in the kernel's type, its FP64 record for the exact near test
// and its vertex ids) and the records of up to 32 trial triangles (rows
// padded by one element against bank conflicts).
template <typename T>
struct FarStage {
    double trec64[TRI_REC];
    T trec[TRI_REC];
    int32_t tv[4];
    T trial[32][TRI_REC + 1];
};

template <int B>
__device__ __forceinline__ void cp_async(void *dst_smem, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"((unsigned)__cvta_generic_to_shared(dst_smem)),
                 "l"(src), "n"(B)
                 : "memory");
}

// Exchanging test and trial triangle transposes a local block, L(s, t) =
// L(t, s)^T, for T (G is symmetric) and for K (the triple product
// f_a . ((r - r') x f_b') keeps its value when r <-> r' and a <-> b), in the
// quadrature too since both triangles use the same 7-point rule.  So the far
// and near stages evaluate and store each unordered pair once, as (t, s) with
// t <= s in the row-major nt x nt planes, and k_mirror fills s < t from it by
// a tiled transpose (component (a, b) of (t, s) is component (b, a) of (s, t)).

// One far (or, by the classification, near -> zero) triangle pair (t, s), t <= s;
// rs is the record of the trial triangle s.
template <typename T>
__device__ __forceinline__ void far_pair(const FarStage<T> &S, int nt, const T *rs,
                                         const double *__restrict__ rec64, const int32_t *__restrict__ vid,
                                         double alpha, const MediaT<T> &md, cx<T> *__restrict__ Zloc, int t, int s) {
    const int64_t plane = (int64_t)nt * nt;
    const int64_t base = (int64_t)t * nt + s;
    int32_t vs[3] = {vid[3 * s], vid[3 * s + 1], vid[3 * s + 2]};
    if (is_near_t<T>(S.trec + TR_CEN, S.trec + TR_CLO, S.trec[TR_H], rs, S.trec64, rec64 + (int64_t)s * TRI_REC, S.tv,
                     vs, alpha)) {
        for (int c = 0; c < NCOMP; ++c) Zloc[c * plane + base] = cx<T>(0, 0);
        return;
    }
    cx<T> out[NCOMP];
    far_entries<T>(S.trec, 1, rs, md, out);
    for (int c = 0; c < NCOMP; ++c) Zloc[c * plane + base] = out[c];
}

// ------------------------------------------------------- near pairs (FP64)
__device__ inline void sub3(const double *a, const double *b, double *c) {
    c[0] = a[0] - b[0]; c[1] = a[1] - b[1]; c[2] = a[2] - b[2];
}
__device__ inline double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
__device__ inline void cross3(const double *a, const double *b, double *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// Closed-form potentials of a flat triangle V at r:
//   I1 = int 1/R, Iv = int (r' - r)/R, I3 = int (r - r')/R^3 (principal value in plane).
// Per edge (Wilton et al. 1984, Graglia 1993): F = ln((R+ + l+)/(R- + l-)) and
// beta = atan(t0 l+ / (R0^2 + |h| R+)) - atan(t0 l- / (R0^2 + |h| R-)).  FP64
// instructions are the cost on this GPU, so each edge takes one logarithm of
// the ratio and one two-argument arctangent of the difference (exact
// identities: atan(n1/d1) - atan(n2/d2) = atan2(n1 d2 - n2 d1, d1 d2 + n1 n2)
// for d1, d2 > 0), normalisations multiply by reciprocal square roots, and the
// distances to the three vertices are formed once.  R + l is taken as
// R0^2 / (R - l) for l < 0 (no cancellation).
__device__ void potentials(const double *V, const double *r, double &I1, double Iv[3], double I3[3]) {
    double e1[3], e2[3], n[3];
    sub3(V + 3, V, e1);
    sub3(V + 6, V, e2);
    cross3(e1, e2, n);
    const double nl2 = dot3(n, n), inl = rsqrt(nl2), nl = nl2 * inl;
    for (int d = 0; d < 3; ++d) n[d] *= inl;
    double rv[3];
    sub3(r, V, rv);
    double h = dot3(n, rv), ah = fabs(h);
    double rho[3] = {r[0] - h * n[0], r[1] - h * n[1], r[2] - h * n[2]};
    double tiny = 1e-28 * nl;
    double Rv[3];   // |r - vertex|
    for (int i = 0; i < 3; ++i) {
        double dv[3];
        sub3(r, V + 3 * i, dv);
        Rv[i] = sqrt(dot3(dv, dv));
    }
    double sum_tF = 0.0, sum_beta = 0.0, vrho[3] = {0, 0, 0}, vF[3] = {0, 0, 0};
    for (int i = 0; i < 3; ++i) {
        const int i1 = (i + 1) % 3;
        const double *A = V + 3 * i, *B = V + 3 * i1;
        double l[3];
        sub3(B, A, l);
        const double ill = rsqrt(dot3(l, l));
        for (int d = 0; d < 3; ++d) l[d] *= ill;
        double u[3];
        cross3(l, n, u);
        double Ar[3], Br[3];
        sub3(A, rho, Ar);
        sub3(B, rho, Br);
        double t0 = dot3(Ar, u), lp = dot3(Br, l), lm = dot3(Ar, l);
        double R02 = t0 * t0 + h * h;
        const double Rp = Rv[i1], Rm = Rv[i];
        double F = 0.0;
        if (R02 > tiny) {   // (R+ + l+)/(R- + l-) as a_n b_d / (a_d b_n)
            const double an = lp >= 0.0 ? Rp + lp : R02, ad = lp >= 0.0 ? 1.0 : Rp - lp;
            const double bn = lm >= 0.0 ? Rm + lm : R02, bd = lm >= 0.0 ? 1.0 : Rm - lm;
            F = log((an * bd) / (ad * bn));
        }
        double beta = 0.0;
        if (ah > 0.0) {
            const double d1 = R02 + ah * Rp, d2 = R02 + ah * Rm;
            beta = atan2(t0 * (lp * d2 - lm * d1), d1 * d2 + t0 * t0 * lp * lm);
        }
        sum_tF += t0 * F;
        sum_beta += beta;
        double cf = 0.5 * (R02 * F + lp * Rp - lm * Rm);
        for (int d = 0; d < 3; ++d) {
            vrho[d] += cf * u[d];
            vF[d] += F * u[d];
        }
    }
    I1 = sum_tF - ah * sum_beta;
    double sg = (h > 0.0) ? 1.0 : ((h < 0.0) ? -1.0 : 0.0);
    for (int d = 0; d < 3; ++d) {
        Iv[d] = vrho[d] - h * n[d] * I1;
        I3[d] = vF[d] + n[d] * sg * sum_beta;
    }
}

// The two smooth remainders of the singularity extraction, from one
// evaluation of e^{-jkR}:
//   gr = (e^{-jkR} - 1)/(4 pi R),                limit -jk/(4 pi) at R = 0
//   hr = g + 1/(4 pi R^3) + k^2/(8 pi R),         limit j k^3/(12 pi) at R = 0
// with g = -(1 + jkR) e^{-jkR}/(4 pi R^3).  For |kR| < 0.2 both come from their
// power series in y = jkR (the direct forms would cancel):
//   gr = -jk/(4 pi)      sum_{j>=0} (-y)^j / (j+1)!
//   hr = -(jk)^3/(4 pi)  sum_{j>=0} (-1)^j (j+2)/(j+3)! y^j
// where 12 terms leave < 1e-19 relative.
__device__ inline void green_rems(z64 k, double R, z64 &gr, z64 &hr) {
    const z64 jk(-k.im, k.re);
    const z64 y = jk * R;
    if (sqrt(norm2(y)) < 0.2) {
        z64 pw(1, 0), s1(0, 0), s2(0, 0);
        double f1 = 1.0, f3 = 6.0;   // (j+1)!, (j+3)!
        for (int j = 0; j < 12; ++j) {
            if (j > 0) {
                pw = pw * y;
                f1 *= (j + 1);
                f3 *= (j + 3);
            }
            const double sg = (j & 1) ? -1.0 : 1.0;
            s1 += (sg / f1) * pw;
            s2 += (sg * (j + 2) / f3) * pw;
        }
        gr = z64(k.im, -k.re) * s1 * (1.0 / (4.0 * PI));
        hr = (jk * jk * jk) * s2 * (-1.0 / (4.0 * PI));
        return;
    }
    double sn, cs;
    sincos(k.re * R, &sn, &cs);
    const double e = exp(k.im * R);
    const z64 ex(e * cs, -e * sn);   // e^{-jkR}
    const double iR = 1.0 / R, i4pR = iR * (1.0 / (4.0 * PI)), i4pR3 = i4pR * iR * iR;
    gr = z64(ex.re - 1.0, ex.im) * i4pR;
    hr = (z64(1, 0) + y) * ex * (-i4pR3) + z64(i4pR3, 0) + (k * k) * (0.5 * i4pR);
}

// One warp per near pair (t <= s).  Lane = 16 o + 8 i + p: orientation o (0:
// test t / trial s, 1: test s / trial t), medium i, test point p < 7 (lane p = 7
// of each group of eight idles).  Each lane forms its test point's
// contribution to the 3 x 3 K and T blocks; groups of eight reduce over p, and
// lane 0 symmetrises, weights the media into Ks, Ta, Tb and stores (t, s).
// FP32 form of the same remainders for the mixed path.  The series branch is
// widened to |kR| < 0.6 so that the direct forms cancel at most a factor
// (kR)^-3 < 5 in single precision; 12 terms leave < 1e-11 relative there.
__device__ inline void green_rems_f(float kre, float kim, float R, c32 &gr, c32 &hr) {
    const float PIf = 3.14159265358979f;
    const c32 jk(-kim, kre);
    const c32 y = jk * R;
    if (sqrtf(y.re * y.re + y.im * y.im) < 0.6f) {
        c32 pw(1, 0), s1(0, 0), s2(0, 0);
        float f1 = 1.0f, f3 = 6.0f;
        for (int j = 0; j < 12; ++j) {
            if (j > 0) {
                pw = pw * y;
                f1 *= (float)(j + 1);
                f3 *= (float)(j + 3);
            }
            const float sg = (j & 1) ? -1.0f : 1.0f;
            s1 += (sg / f1) * pw;
            s2 += (sg * (float)(j + 2) / f3) * pw;
        }
        gr = c32(kim, -kre) * s1 * (1.0f / (4.0f * PIf));
        hr = (jk * jk * jk) * s2 * (-1.0f / (4.0f * PIf));
        return;
    }
    float sn, cs;
    sincosf(kre * R, &sn, &cs);
    const float e = expf(kim * R);
    const c32 ex(e * cs, -e * sn);
    const float iR = 1.0f / R, i4pR = iR * (1.0f / (4.0f * PIf)), i4pR3 = i4pR * iR * iR;
    gr = c32(ex.re - 1.0f, ex.im) * i4pR;
    hr = (c32(1, 0) + y) * ex * (-i4pR3) + c32(i4pR3, 0) + (c32(kre, kim) * c32(kre, kim)) * (0.5f * i4pR);
}

// Near pairs, two per warp.  Lane = 16 slot + 8 o + p: pair slot (0, 1),
// orientation o (0: test t / trial s, 1: test s / trial t), test point p < 7
// (lane p = 7 of each group of eight idles).  Each lane evaluates the closed-
// form potentials of the trial triangle at its test point once, then for both
// media adds the bounded remainders and forms its weighted share of the test-
// point moments, with r relative to the test triangle's centroid:
//   M0 = sum w S0, Mr0 = sum w r S0, Mrr0 = sum w |r|^2 S0, MS = sum w Sr,
//   MrS = sum w r.Sr, MW = sum w Wv, MX = sum w Wv x r.
// Expanding the bilinear point terms in r gives the 3 x 3 entries from the
// moments (P = test vertex a, Q = trial vertex b, both relative):
//   T~_ab = c_a d_b (-jk) [MrS - P.MS + Mrr0 - (P + Q).Mr0 + (P.Q - 4/k^2) M0]
//   K~_ab = c_a d_b [(Q - P).MX + P.(MW x Q)]        (0 when t = s)
// The moments are summed over the 7 test points by shuffles and staged in
// shared memory; lanes (slot, a, b) then symmetrise, weight the media into
// Ks, Ta, Tb and store (t, s), t <= s (the (s, t) block is its transpose).
constexpr int NEAR_MOM = 15;   // complex moments per (orientation, medium)

// Work of one near pair, counted from the operations of near_pair2 with each
// square root, logarithm, arctangent, sine/cosine pair and exponential as one:
// per orientation and test point (14 lanes) the closed-form potentials of the
// trial triangle (3 edges x 50 + 40, the vertex distances formed once), the
// trial-point geometry (7 x 10) and their sums into S0, Sr, Wv (2 media x 12),
// FP64 on both paths; the outer quadrature, FP64 on the FP64 path and FP32 on
// the mixed one: for each medium the 15 test-point moments (90), their
// reductions (15 complex x 2 media x 3 shuffle steps on 16 lanes) and the 9
// entries (2 orientations x 2 media x 60); and the 7 remainder evaluations with
// their weighted sums per medium (7 x 60), likewise.
constexpr double NEAR_FP64_OPS_CLOSED = 14 * (190 + 70 + 2 * 12);
constexpr double NEAR_OUTER_OPS = 14 * 2 * 90 + 16 * 15 * 2 * 3 * 2 + 9 * 2 * 2 * 60;
constexpr double NEAR_REM_OPS = 14 * 2 * 7 * 60;
// FP64 operations per near pair of the near-pair kernel in type T
template <typename T>
constexpr double near_fp64_ops() {
    return NEAR_FP64_OPS_CLOSED + (sizeof(T) == 8 ? NEAR_OUTER_OPS + NEAR_REM_OPS : 0.0);
}

template <typename T>
__device__ __forceinline__ void near_pair2(int t, int s, int nt, const double *__restrict__ rec, const Media &md,
                                           cx<T> *__restrict__ Zloc, cx<T> (*sm)[2][2][NEAR_MOM],
                                           cx<T> *__restrict__ blk = nullptr) {
    // (t, s): the pair of this lane's slot (t < 0: none); every lane reads only
    // its own slot's mesh, and all 32 lanes reach the shuffles and barriers
    const int lane = threadIdx.x & 31;
    const int slot = lane >> 4, o = (lane >> 3) & 1, p = lane & 7;
    __syncwarp();   // the slot's previous readers are done
    // the test-point moments and the entries are the outer quadrature of the
    // closed forms: in T (FP32 on the mixed path, like the remainders)
    cx<T> mom[2][NEAR_MOM];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int c = 0; c < NEAR_MOM; ++c) mom[i][c] = cx<T>(0, 0);
    if (p < 7 && t >= 0) {
        const double *A = rec + (int64_t)(o == 0 ? t : s) * TRI_REC;
        const double *B = rec + (int64_t)(o == 0 ? s : t) * TRI_REC;
        const double *r = A + TR_Q + 3 * p;
        double I1, Iv[3], I3[3];
        potentials(B + TR_P, r, I1, Iv, I3);
        const T wp = (T)A[TR_W + p];
        const T rr[3] = {(T)(r[0] - A[TR_CEN]), (T)(r[1] - A[TR_CEN + 1]), (T)(r[2] - A[TR_CEN + 2])};
        const T r2 = rr[0] * rr[0] + rr[1] * rr[1] + rr[2] * rr[2];
        // trial points: d = r - r', R, weights; shared by the two media.  On the
        // mixed path the smooth remainders, their 7-point sums and the moments
        // are FP32 and only the closed forms FP64.
        T dq[7][3], Rq[7], wq[7];
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            double dv[3];
            sub3(r, B + TR_Q + 3 * q, dv);
            for (int d = 0; d < 3; ++d) dq[q][d] = (T)dv[d];
            if constexpr (sizeof(T) == 4) Rq[q] = sqrtf(dq[q][0] * dq[q][0] + dq[q][1] * dq[q][1] + dq[q][2] * dq[q][2]);
            else Rq[q] = sqrt(dot3(dv, dv));
            wq[q] = (T)B[TR_W + q];
        }
#pragma unroll
        for (int med = 0; med < 2; ++med) {
            const z64 k = med == 0 ? z64(md.k1r, md.k1i) : z64(md.k2r, md.k2i);
            const z64 kk = k * k;
            cx<T> g0(0, 0), gr[3], hw[3];   // sum w g, sum w g (-d), sum w h d over the trial points
            for (int d = 0; d < 3; ++d) gr[d] = hw[d] = cx<T>(0, 0);
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                cx<T> gs, hs;
                if constexpr (sizeof(T) == 4) {
                    green_rems_f((float)k.re, (float)k.im, Rq[q], gs, hs);
                } else {
                    green_rems(k, Rq[q], gs, hs);
                }
                gs = gs * wq[q];
                hs = hs * wq[q];
                g0 += gs;
                for (int d = 0; d < 3; ++d) {
                    gr[d] += gs * (-dq[q][d]);
                    hw[d] += hs * dq[q][d];
                }
            }
            const cx<T> S0((T)(I1 / (4.0 * PI)) + g0.re, g0.im);
            cx<T> Sr[3], Wv[3];
            for (int d = 0; d < 3; ++d) {
                Sr[d] = cx<T>((T)(Iv[d] / (4.0 * PI)) + gr[d].re, gr[d].im);
                const z64 kI = kk * (Iv[d] / (8.0 * PI));
                Wv[d] = cx<T>((T)(kI.re - I3[d] / (4.0 * PI)), (T)kI.im) + hw[d];
            }
            cx<T> *m = mom[med];
            const cx<T> wS0 = wp * S0;
            m[0] = wS0;
            m[1] = rr[0] * wS0; m[2] = rr[1] * wS0; m[3] = rr[2] * wS0;
            m[4] = r2 * wS0;
            m[5] = wp * Sr[0]; m[6] = wp * Sr[1]; m[7] = wp * Sr[2];
            m[8] = rr[0] * m[5] + rr[1] * m[6] + rr[2] * m[7];
            m[9] = wp * Wv[0]; m[10] = wp * Wv[1]; m[11] = wp * Wv[2];
            // Wv x r
            m[12] = rr[2] * m[10] - rr[1] * m[11];
            m[13] = rr[0] * m[11] - rr[2] * m[9];
            m[14] = rr[1] * m[9] - rr[0] * m[10];
        }
    }
    // sum over the eight lanes of each (slot, o) group
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int c = 0; c < NEAR_MOM; ++c)
#pragma unroll
            for (int off = 1; off < 8; off <<= 1) {
                mom[i][c].re += __shfl_xor_sync(0xffffffffu, mom[i][c].re, off);
                mom[i][c].im += __shfl_xor_sync(0xffffffffu, mom[i][c].im, off);
            }
    if (p == 0)
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int c = 0; c < NEAR_MOM; ++c) sm[slot][o][i][c] = mom[i][c];
    __syncwarp();
    const int e = lane & 15;
    if (e >= 9 || t < 0) return;
    // lane (slot, e = 3 a + b): entry (a, b) of (t, s) = 1/2 [L~_o0(a, b) + L~_o1(b, a)]
    const int a = e / 3, b = e % 3;
    cx<T> ks(0, 0), ta(0, 0), tb(0, 0);
#pragma unroll
    for (int oo = 0; oo < 2; ++oo) {
        const double *A = rec + (int64_t)(oo == 0 ? t : s) * TRI_REC;
        const double *B = rec + (int64_t)(oo == 0 ? s : t) * TRI_REC;
        const int ia = oo == 0 ? a : b, ib = oo == 0 ? b : a;   // test vertex, trial vertex
        T P[3], Q[3];
        for (int d = 0; d < 3; ++d) {
            P[d] = (T)(A[TR_P + 3 * ia + d] - A[TR_CEN + d]);
            Q[d] = (T)(B[TR_P + 3 * ib + d] - A[TR_CEN + d]);
        }
        const T cc = (T)(0.5 * A[TR_C + ia] * B[TR_C + ib]);
        const T PQ = P[0] * Q[0] + P[1] * Q[1] + P[2] * Q[2];
        const T PpQ[3] = {P[0] + Q[0], P[1] + Q[1], P[2] + Q[2]};
        const T QmP[3] = {Q[0] - P[0], Q[1] - P[1], Q[2] - P[2]};
        // P x Q: P.(MW x Q) = MW.(Q x P)
        const T QxP[3] = {Q[1] * P[2] - Q[2] * P[1], Q[2] * P[0] - Q[0] * P[2], Q[0] * P[1] - Q[1] * P[0]};
#pragma unroll
        for (int med = 0; med < 2; ++med) {
            const cx<T> *m = sm[slot][oo][med];
            const cx<T> k = med == 0 ? cx<T>((T)md.k1r, (T)md.k1i) : cx<T>((T)md.k2r, (T)md.k2i);
            const cx<T> eta = med == 0 ? cx<T>((T)md.e1r, (T)md.e1i) : cx<T>((T)md.e2r, (T)md.e2i);
            const cx<T> f4k2 = med == 0 ? cx<T>((T)md.f1r, (T)md.f1i) : cx<T>((T)md.f2r, (T)md.f2i);   // 4 / k^2
            const cx<T> ieta = med == 0 ? cx<T>((T)md.i1r, (T)md.i1i) : cx<T>((T)md.i2r, (T)md.i2i);   // 1 / eta
            cx<T> br = m[8] + m[4] - (P[0] * m[5] + P[1] * m[6] + P[2] * m[7]) -
                       (PpQ[0] * m[1] + PpQ[1] * m[2] + PpQ[2] * m[3]) + PQ * m[0] - f4k2 * m[0];
            const cx<T> Tv = cc * (cx<T>(k.im, -k.re) * br);
            ta += -eta * Tv;
            tb += Tv * ieta;
            if (t != s)
                ks += cc * (QmP[0] * m[12] + QmP[1] * m[13] + QmP[2] * m[14] + QxP[0] * m[9] + QxP[1] * m[10] +
                            QxP[2] * m[11]);
        }
    }
    const cx<T> v[3] = {ks, ta, tb};
    const int64_t plane = (int64_t)nt * nt;
    for (int op = 0; op < 3; ++op) {
        const cx<T> val = v[op];
        if (blk) {   // compact form: the (t, s) block of this pair; (s, t) is its transpose
            blk[op * 9 + 3 * a + b] = val;
            continue;
        }
        Zloc[(op * 9 + 3 * a + b) * plane + (int64_t)t * nt + s] = val;   // t <= s; (s, t) by k_mirror
    }
}

// ------------------------------------------------ several meshes at once
// One job per mesh; the batch kernels flatten the meshes' work items and find
// the job of an item by binary search over the jobs' first item.
template <typename T>
struct AsmJob {
    const T *rec;
    const double *rec64;
    const int32_t *vid, *pairs, *edge_tri, *edge_loc;
    const int32_t *tri_cell;   // non-null: evaluate only pairs of triangles that share a cell
    cx<T> *Zloc, *Z;
    cx<T> *nearblk;            // non-null: near-pair blocks in compact form, 27 per pair of the near list
    MediaT<T> mdt;
    Media md;
    double alpha;
    int nt, strip, nstrip;   // far tasks: trial triangles per task (multiple of 32), tasks per test triangle
    int64_t ne, far0, near0, row0, mir0;   // first far task, near pair, gather row and mirror tile of the job
};

template <typename T, int64_t AsmJob<T>::*F>
__device__ __forceinline__ int find_job(const AsmJob<T> *jobs, int njobs, int64_t item) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].*F <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ bool share_cell(const int32_t *__restrict__ tc, int t, int s) {
    const int a0 = tc[3 * t], a1 = tc[3 * t + 1], a2 = tc[3 * t + 2];
    bool r = false;
    for (int k = 0; k < 3; ++k) {
        const int b = tc[3 * s + k];
        r |= (b == a0) | (b == a1) | (b == a2);
    }
    return r;
}

// Far pairs of all meshes: persistent warps take tasks (mesh, test triangle,
// strip of trial triangles) from an atomic counter, so meshes of uneven size
// share the GPU without a tail per mesh.  A warp works through its task 32
// trial triangles at a time; each item (test triangle and 32 trial records)
// is staged in the warp's own shared memory by asynchronous copies, the next
// item (the task's next 32, or the first 32 of a newly taken task) while the
// current one is computed, so warps never wait on one another and rarely on
// memory.
template <typename T>
__host__ __device__ constexpr int far_warps() { return sizeof(T) == 4 ? 4 : 2; }
template <typename T>
constexpr size_t far_smem() { return (size_t)2 * far_warps<T>() * sizeof(FarStage<T>); }

template <typename T>
__device__ __forceinline__ void far_stage(FarStage<T> &S, const AsmJob<T> &J, int t, int s0, int cnt, int lane) {
    for (int i = lane; i < TRI_REC; i += 32) {
        cp_async<sizeof(T)>(&S.trec[i], J.rec + (int64_t)t * TRI_REC + i);
        cp_async<8>(&S.trec64[i], J.rec64 + (int64_t)t * TRI_REC + i);
    }
    if (lane < 3) cp_async<4>(&S.tv[lane], J.vid + 3 * (int64_t)t + lane);
    const T *src = J.rec + (int64_t)s0 * TRI_REC;
#pragma unroll 4
    for (int idx = lane; idx < cnt * TRI_REC; idx += 32)
        cp_async<sizeof(T)>(&S.trial[idx / TRI_REC][idx % TRI_REC], src + idx);
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Far tasks of a job before test-triangle block i (blocks of one strip width,
// block i taking the strips i .. nstrip - 1), and in the whole job.
template <typename T>
__host__ __device__ __forceinline__ int64_t far_before(const AsmJob<T> &J, int i) {
    return (int64_t)J.strip * ((int64_t)i * J.nstrip - ((int64_t)i * (i - 1)) / 2);
}
template <typename T>
int64_t far_tasks(const AsmJob<T> &J) {
    const int last = J.nstrip - 1;
    return far_before(J, last) + (int64_t)(J.nt - last * J.strip);
}

// FP32: three blocks of four warps per SM (168 registers) for more warps in
// flight; FP64: four blocks of two warps, where the wider accumulators would
// otherwise spill.
template <typename T>
__global__ void __launch_bounds__(32 * far_warps<T>(), sizeof(T) == 4 ? 3 : 4)
    k_far(const AsmJob<T> *__restrict__ jobs, int njobs, int64_t ntasks, unsigned long long *__restrict__ counter) {
    extern __shared__ __align__(16) unsigned char far_raw[];
    const int lane = threadIdx.x & 31;
    FarStage<T> *stage = reinterpret_cast<FarStage<T> *>(far_raw) + 2 * (threadIdx.x >> 5);
    // the task being staged: job, test triangle, end of its strip
    int tj = 0, tt = 0, tse = 0;
    auto grab = [&](int &s0) -> bool {
        unsigned long long task = 0;
        if (lane == 0) task = atomicAdd(counter, 1ull);
        task = __shfl_sync(0xffffffffu, task, 0);
        if ((int64_t)task >= ntasks) return false;
        tj = find_job<T, &AsmJob<T>::far0>(jobs, njobs, (int64_t)task);
        const AsmJob<T> &J = jobs[tj];
        const int64_t local = (int64_t)task - J.far0;
        // upper triangle: the test triangles in blocks of one strip width W; block i
        // takes the strips i .. nstrip - 1 for each of its test triangles, and the
        // blocks before it hold far_before(i) = W (i nstrip - i (i - 1) / 2) tasks
        int lo = 0, hi = J.nstrip - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (far_before(J, mid) <= local) lo = mid;
            else hi = mid - 1;
        }
        const int64_t l2 = local - far_before(J, lo);
        const int per = J.nstrip - lo;
        tt = lo * J.strip + (int)(l2 / per);
        s0 = (lo + (int)(l2 % per)) * J.strip;
        tse = min(s0 + J.strip, J.nt);
        s0 = max(s0, tt & ~31);   // on the diagonal strip, from the 32 trial triangles holding s = t
        return true;
    };
    int cs0 = 0;
    if (!grab(cs0)) return;
    int cj = tj, ct = tt, ccnt = min(32, tse - cs0);
    far_stage(stage[0], jobs[cj], ct, cs0, ccnt, lane);
    for (int b = 0;; b ^= 1) {
        int ns0 = cs0 + 32;
        bool more = ns0 < tse;
        if (!more) more = grab(ns0);
        const int nj = tj, nt_ = tt, ncnt = more ? min(32, tse - ns0) : 0;
        if (more) {
            far_stage(stage[b ^ 1], jobs[nj], nt_, ns0, ncnt, lane);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncwarp();
        {
            const AsmJob<T> &J = jobs[cj];
            const int s = cs0 + lane;
            if (lane < ccnt && s >= ct) {
                if (J.tri_cell && !share_cell(J.tri_cell, ct, s)) {
                    const int64_t plane = (int64_t)J.nt * J.nt, base = (int64_t)ct * J.nt + s;
                    for (int c = 0; c < NCOMP; ++c) J.Zloc[c * plane + base] = cx<T>(0, 0);
                } else {
                    far_pair(stage[b], J.nt, stage[b].trial[lane], J.rec64, J.vid, J.alpha, J.mdt, J.Zloc, ct, s);
                }
            }
        }
        __syncwarp();   // the stage is restaged two items later
        if (!more) break;
        cj = nj;
        ct = nt_;
        cs0 = ns0;
        ccnt = ncnt;
    }
}

// Near pairs of all meshes: two pairs per warp (the pairs of one warp may
// belong to different meshes), grid-stride over pair couples.
template <typename T>
__global__ void __launch_bounds__(128) k_near_blocks(const AsmJob<T> *__restrict__ jobs, int njobs, int64_t npairs) {
    __shared__ cx<T> sm_all[4][2][2][2][NEAR_MOM];
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t ncouple = (npairs + 1) / 2;
    const int slot = (threadIdx.x >> 4) & 1;
    for (int64_t cp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; cp < ncouple; cp += nw) {
        const int64_t pid = 2 * cp + slot;
        int t = -1, s = -1;
        const AsmJob<T> *J = &jobs[0];
        if (pid < npairs) {
            J = &jobs[find_job<T, &AsmJob<T>::near0>(jobs, njobs, pid)];
            const int64_t l = pid - J->near0;
            t = J->pairs[2 * l];
            s = J->pairs[2 * l + 1];
            if (J->tri_cell && !share_cell(J->tri_cell, t, s)) t = s = -1;   // stays zero (written by k_far)
        }
        cx<T> *blk = (J->nearblk && t >= 0) ? J->nearblk + (pid - J->near0) * NCOMP : nullptr;
        near_pair2<T>(t, s, J->nt, J->rec64, J->md, J->Zloc, sm_all[(threadIdx.x >> 5) & 3], blk);
    }
}

// The blocks of the pairs s < t of all meshes from the stored (s, t): one
// TM x TM tile of one component plane per CTA (TM x 256/TM threads; TM = 64
// complex64 or 32 complex128 entries, 512-byte row segments), read along the
// rows of (s, t) and written along the rows of (t, s) through shared memory;
// the tiles of a mesh are those on and below the diagonal, tile l = (bi, bj)
// with l = bi (bi + 1) / 2 + bj, and component (a, b) of (t, s) comes from
// component (b, a) of (s, t).
template <typename T>
__host__ __device__ constexpr int mir_tile() { return sizeof(T) == 4 ? 64 : 32; }

template <typename T>
__global__ void __launch_bounds__(256) k_mirror(const AsmJob<T> *__restrict__ jobs, int njobs, int64_t ntiles) {
    constexpr int TM = mir_tile<T>(), TY = 256 / TM;
    __shared__ cx<T> tile[TM][TM + 1];
    const int c = blockIdx.y;   // destination component op * 9 + 3 a + b
    const int csrc = (c / 9) * 9 + 3 * (c % 3) + (c % 9) / 3;
    const int tx = threadIdx.x % TM, ty = threadIdx.x / TM;
    for (int64_t l = blockIdx.x; l < ntiles; l += gridDim.x) {
        const AsmJob<T> &J = jobs[find_job<T, &AsmJob<T>::mir0>(jobs, njobs, l)];
        const int64_t loc = l - J.mir0;
        // FP32 estimate (FP64 issue is scarce here), corrected to the exact row by the loops
        int64_t bi = (int64_t)((sqrtf(8.0f * (float)loc + 1.0f) - 1.0f) * 0.5f);
        while ((bi + 1) * (bi + 2) / 2 <= loc) ++bi;
        while (bi * (bi + 1) / 2 > loc) --bi;
        const int t0 = (int)bi * TM, s0 = (int)(loc - bi * (bi + 1) / 2) * TM;   // destination rows t, columns s
        const int nt = J.nt;
        const int64_t plane = (int64_t)nt * nt;
        const cx<T> *src = J.Zloc + (int64_t)csrc * plane;
        cx<T> *dst = J.Zloc + (int64_t)c * plane;
        const int tc = t0 + tx;
#pragma unroll
        for (int y = ty; y < TM; y += TY) {   // tile[y][x] = (s0 + y, t0 + x) of the source
            const int sr = s0 + y;
            if (tc < nt && sr < tc) tile[y][tx] = src[(int64_t)sr * nt + tc];
        }
        __syncthreads();
        const int sc = s0 + tx;
#pragma unroll
        for (int y = ty; y < TM; y += TY) {   // (t0 + y, s0 + x) = source (s0 + x, t0 + y)
            const int tr = t0 + y;
            if (tr < nt && sc < tr) dst[(int64_t)tr * nt + sc] = tile[tx][y];
        }
        __syncthreads();
    }
}

// Gather of all meshes: one block per RWG row, grid-stride over the rows of all meshes.
template <typename T>
__global__ void k_gather(const AsmJob<T> *__restrict__ jobs, int njobs, int64_t nrows) {
    for (int64_t row = blockIdx.x; row < nrows; row += gridDim.x) {
        const AsmJob<T> &J = jobs[find_job<T, &AsmJob<T>::row0>(jobs, njobs, row)];
        const int64_t i = row - J.row0, ne = J.ne;
        const int64_t plane = (int64_t)J.nt * J.nt;
        const int ti[2] = {J.edge_tri[2 * i], J.edge_tri[2 * i + 1]}, ai[2] = {J.edge_loc[2 * i], J.edge_loc[2 * i + 1]};
        for (int64_t j = threadIdx.x; j < ne; j += blockDim.x) {
            const int tj[2] = {J.edge_tri[2 * j], J.edge_tri[2 * j + 1]};
            const int aj[2] = {J.edge_loc[2 * j], J.edge_loc[2 * j + 1]};
            for (int op = 0; op < 3; ++op) {
                cx<T> v(0, 0);
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b)
                        v += J.Zloc[(op * 9 + 3 * ai[a] + aj[b]) * plane + (int64_t)ti[a] * J.nt + tj[b]];
                J.Z[(op * ne + i) * ne + j] = v;
            }
        }
    }
}

}  // namespace

template <typename T>
void assemble_rwg_batch(const std::vector<Mesh *> &ms, const std::vector<cx<T> *> &Z, cudaStream_t st,
                        bool diag_cells);

// One mesh: the batched stages with a batch of one (one code path, so a
// mesh assembled alone and in a batch gets the same bits).
template <typename T>
void assemble_rwg(Mesh &m, cx<T> *Zrwg, cudaStream_t st, bool diag_cells) {
    assemble_rwg_batch<T>(std::vector<Mesh *>{&m}, std::vector<cx<T> *>{Zrwg}, st, diag_cells);
}

template void assemble_rwg<double>(Mesh &, z64 *, cudaStream_t, bool);
template void assemble_rwg<float>(Mesh &, c32 *, cudaStream_t, bool);
// Local blocks, far/near pairs and RWG gather of several meshes, one launch
// per stage.  The far stage's strip width (trial triangles per task) is
// picked once per device and precision by timing the candidates, twice each,
// on the first batch (every candidate writes the same values, so the batch
// is not run again afterwards).
template <typename T>
void assemble_rwg_batch(const std::vector<Mesh *> &ms, const std::vector<cx<T> *> &Z, cudaStream_t st,
                        bool diag_cells) {
    const int nj = (int)ms.size();
    if (nj == 0) return;
    std::vector<DevBuf<cx<T>>> Zloc(nj);
    std::vector<AsmJob<T>> jobs(nj);
    int64_t npairs = 0, nrows = 0, ntiles = 0;
    double far_flop = 0.0, far_bytes = 0.0, mir_bytes = 0.0, gat_bytes = 0.0;
    for (int k = 0; k < nj; ++k) {
        Mesh &m = *ms[k];
        const int nt = (int)m.h.nt;
        Zloc[k].alloc((size_t)NCOMP * nt * nt);
        const Media md = media_full(m.k1, m.k2, m.eta1, m.eta2);
        AsmJob<T> &J = jobs[k];
        if constexpr (sizeof(T) == 8) J.rec = (const T *)m.tri64.p;
        else J.rec = (const T *)m.tri32.p;
        J.rec64 = m.tri64.p;
        J.vid = m.tri_vid.p;
        J.pairs = m.near_pairs.p;
        J.edge_tri = m.edge_tri.p;
        J.edge_loc = m.edge_loc.p;
        J.tri_cell = diag_cells ? m.tri_cell.p : nullptr;
        J.Zloc = Zloc[k].p;
        J.Z = Z[k];
        J.mdt = media_t<T>(md);
        J.md = md;
        J.alpha = m.alpha;
        J.nt = nt;
        J.ne = m.h.ne;
        J.near0 = npairs;
        J.row0 = nrows;
        J.mir0 = ntiles;
        npairs += m.n_near;
        nrows += m.h.ne;
        const int64_t tb = (nt + mir_tile<T>() - 1) / mir_tile<T>();
        ntiles += tb * (tb + 1) / 2;
        mir_bytes += 2.0 * NCOMP * (0.5 * nt * (nt - 1.0)) * sizeof(cx<T>);   // pairs s < t read and written
        // the gather reads every local block once and writes the three RWG planes
        gat_bytes += ((double)NCOMP * nt * nt + 3.0 * (double)m.h.ne * m.h.ne) * sizeof(cx<T>);
        const double upper = 0.5 * nt * (nt + 1.0);   // pairs t <= s
        far_flop += (upper - (double)m.n_near) * 49.0 * FAR_FLOP_PER_POINT_PAIR;
        far_bytes += (double)NCOMP * upper * sizeof(cx<T>);
    }
    int dev = 0, nsm = 0;
    CBFM_CUDA(cudaGetDevice(&dev));
    CBFM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    DevBuf<AsmJob<T>> djobs;
    djobs.alloc(nj);
    DevBuf<unsigned long long> counter;
    counter.alloc(1);
    const std::string key = std::string("far_strip_") + (sizeof(T) == 8 ? "f64" : "f32") + "_dev" + std::to_string(dev);
    int tuned = tuning_get(key);
    const std::vector<int> cands = tuned > 0 ? std::vector<int>{tuned} : std::vector<int>{32, 64, 128};
    std::vector<float> t_ms(cands.size(), 1e30f);
    // while tuning, every candidate runs twice (the faster run counts) so that
    // a first-launch delay or one noisy timing does not decide
    const int reps = tuned > 0 ? 1 : 2;
    for (int rep = 0; rep < reps; ++rep)
    for (size_t ci = 0; ci < cands.size(); ++ci) {
        const int W = cands[ci];
        int64_t ntask = 0;
        for (auto &J : jobs) {
            J.strip = W;
            J.nstrip = (J.nt + W - 1) / W;
            J.far0 = ntask;
            ntask += far_tasks(J);
        }
        CBFM_CUDA(cudaMemcpyAsync(djobs.p, jobs.data(), sizeof(AsmJob<T>) * nj, cudaMemcpyHostToDevice, st));
        CBFM_CUDA(cudaMemsetAsync(counter.p, 0, sizeof(unsigned long long), st));
        constexpr int FB = 32 * far_warps<T>();
        CBFM_CUDA(cudaFuncSetAttribute(k_far<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)far_smem<T>()));
        int occ = 0;
        CBFM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_far<T>, FB, far_smem<T>()));
        const unsigned grid = (unsigned)std::max(1, occ) * (unsigned)nsm;
        cudaEvent_t e0, e1;
        CBFM_CUDA(cudaEventCreate(&e0));
        CBFM_CUDA(cudaEventCreate(&e1));
        CBFM_CUDA(cudaEventRecord(e0, st));
        {
            ProfScope ps_("k_far", st);
            k_far<T><<<grid, FB, far_smem<T>(), st>>>(djobs.p, nj, ntask, counter.p);
            launched("k_far");
        }
        CBFM_CUDA(cudaEventRecord(e1, st));
        CBFM_CUDA(cudaEventSynchronize(e1));
        float ms_ = 0.f;
        CBFM_CUDA(cudaEventElapsedTime(&ms_, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        t_ms[ci] = std::min(t_ms[ci], ms_);
    }
    if (tuned <= 0) {
        size_t bi = 0;
        for (size_t ci = 1; ci < cands.size(); ++ci)
            if (t_ms[ci] < t_ms[bi]) bi = ci;
        tuning_set(key, cands[bi]);
    }
    prof_add_work("k_far", far_flop, far_bytes);
    prof_add_work("k_near_blocks", (double)npairs * near_fp64_ops<T>(),
                  (double)npairs * (2 * TRI_REC * sizeof(double) + 27 * sizeof(cx<T>)));
    if (npairs > 0) {
        int occ = 0;
        CBFM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_near_blocks<T>, 128, 0));
        const unsigned grid = (unsigned)std::min<int64_t>((int64_t)std::max(1, occ) * nsm, ((npairs + 1) / 2 * 32 + 127) / 128);
        ProfScope ps_("k_near_blocks", st);
        k_near_blocks<T><<<grid, 128, 0, st>>>(djobs.p, nj, npairs);
        launched("k_near_blocks");
    }
    {
        const dim3 grid((unsigned)std::min<int64_t>(ntiles, 1 << 20), NCOMP);
        prof_add_work("k_mirror", 0.0, mir_bytes);
        ProfScope ps_("k_mirror", st);
        k_mirror<T><<<grid, 256, 0, st>>>(djobs.p, nj, ntiles);
        launched("k_mirror");
    }
    {
        const unsigned grid = (unsigned)std::min<int64_t>(nrows, 8 * (int64_t)nsm);
        prof_add_work("k_gather", 0.0, gat_bytes);
        ProfScope ps_("k_gather", st);
        k_gather<T><<<grid, 128, 0, st>>>(djobs.p, nj, nrows);
        launched("k_gather");
    }
    CBFM_CUDA(cudaStreamSynchronize(st));   // the local blocks are released on return
}

// The near-pair stage alone, in compact form: out[k][27 l + c] is component c
// (op x 3 x 3) of the (t, s) block of near pair l of mesh k (FP64 closed forms;
// smooth remainders in T).  One launch over all meshes.
template <typename T>
void near_blocks_compact_t(const std::vector<Mesh *> &ms, const std::vector<cx<T> *> &out, cudaStream_t st) {
    const int nj = (int)ms.size();
    std::vector<AsmJob<T>> jobs(nj);
    int64_t npairs = 0;
    for (int k = 0; k < nj; ++k) {
        Mesh &m = *ms[k];
        AsmJob<T> &J = jobs[k];
        J = AsmJob<T>{};
        if constexpr (sizeof(T) == 8) J.rec = (const T *)m.tri64.p;
        else J.rec = (const T *)m.tri32.p;
        J.rec64 = m.tri64.p;
        J.vid = m.tri_vid.p;
        J.pairs = m.near_pairs.p;
        J.nearblk = out[k];
        J.md = media_full(m.k1, m.k2, m.eta1, m.eta2);
        J.mdt = media_t<T>(J.md);
        J.alpha = m.alpha;
        J.nt = (int)m.h.nt;
        J.ne = m.h.ne;
        J.near0 = npairs;
        npairs += m.n_near;
    }
    if (npairs == 0) return;
    DevBuf<AsmJob<T>> djobs;
    djobs.alloc(nj);
    CBFM_CUDA(cudaMemcpyAsync(djobs.p, jobs.data(), sizeof(AsmJob<T>) * nj, cudaMemcpyHostToDevice, st));
    int occ = 0;
    CBFM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_near_blocks<T>, 128, 0));
    const unsigned grid =
        (unsigned)std::min<int64_t>((int64_t)std::max(1, occ) * sm_count(), ((npairs + 1) / 2 * 32 + 127) / 128);
    prof_add_work("k_near_blocks", (double)npairs * near_fp64_ops<T>(),
                  (double)npairs * (2 * TRI_REC * sizeof(double) + 27 * sizeof(cx<T>)));
    {
        ProfScope ps_("k_near_blocks", st);
        k_near_blocks<T><<<grid, 128, 0, st>>>(djobs.p, nj, npairs);
        launched("k_near_blocks");
    }
    CBFM_CUDA(cudaStreamSynchronize(st));   // djobs is released on return
}

template void near_blocks_compact_t<float>(const std::vector<Mesh *> &, const std::vector<c32 *> &, cudaStream_t);
template void near_blocks_compact_t<double>(const std::vector<Mesh *> &, const std::vector<z64 *> &, cudaStream_t);

void near_blocks_compact(const std::vector<Mesh *> &ms, const std::vector<c32 *> &out, cudaStream_t st) {
    near_blocks_compact_t<float>(ms, out, st);
}

template void assemble_rwg_batch<double>(const std::vector<Mesh *> &, const std::vector<z64 *> &, cudaStream_t, bool);
template void assemble_rwg_batch<float>(const std::vector<Mesh *> &, const std::vector<c32 *> &, cudaStream_t, bool);

}  // namespace cbfm
