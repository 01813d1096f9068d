// k_geom.cu -- geometry staging, near-pair list, RWG Gram rows, plane-wave
// right-hand sides and far field (paper Sec. II-B; Sec. III-B Eq. (gram_RWG);
// Eq. (v); monostatic/bistatic RCS after Knott).
#include <vector>

#include "internal.cuh"

namespace cbfm {

namespace {

// 7-point degree-5 rule (Radon): centroid weight 9/40 and two 3-point orbits
// (a, b, b) with b = (6 -/+ sqrt 15)/21, weights (155 -/+ sqrt 15)/1200.
__device__ void quad7(double bary[7][3], double w[7]) {
    const double s15 = sqrt(15.0);
    const double b1 = (6.0 - s15) / 21.0, a1 = 1.0 - 2.0 * b1;
    const double b2 = (6.0 + s15) / 21.0, a2 = 1.0 - 2.0 * b2;
    const double w1 = (155.0 - s15) / 1200.0, w2 = (155.0 + s15) / 1200.0;
    const double B[7][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3}, {a1, b1, b1}, {b1, a1, b1}, {b1, b1, a1},
                            {a2, b2, b2}, {b2, a2, b2}, {b2, b2, a2}};
    const double W[7] = {9.0 / 40.0, w1, w1, w1, w2, w2, w2};
    for (int p = 0; p < 7; ++p) {
        w[p] = W[p];
        for (int k = 0; k < 3; ++k) bary[p][k] = B[p][k];
    }
}

// |x| with separately rounded products/sums (no FMA contraction), so the
// near classification is reproducible bit for bit.
__device__ inline double norm3_rn(double x, double y, double z) {
    return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z)));
}

__global__ void k_tri_records(int64_t nt, const double *__restrict__ V, const int32_t *__restrict__ tris,
                              const int32_t *__restrict__ tri_edge, const int32_t *__restrict__ tri_sign,
                              const double *__restrict__ edge_len, double cx, double cy, double cz,
                              double *__restrict__ rec64, float *__restrict__ rec32) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    double v[3][3];
    for (int a = 0; a < 3; ++a)
        for (int d = 0; d < 3; ++d) v[a][d] = V[3 * tris[3 * t + a] + d];
    double e1[3], e2[3], e3[3];
    for (int d = 0; d < 3; ++d) {
        e1[d] = __dsub_rn(v[1][d], v[0][d]);
        e2[d] = __dsub_rn(v[2][d], v[0][d]);
        e3[d] = __dsub_rn(v[2][d], v[1][d]);
    }
    double n0 = e1[1] * e2[2] - e1[2] * e2[1];
    double n1 = e1[2] * e2[0] - e1[0] * e2[2];
    double n2 = e1[0] * e2[1] - e1[1] * e2[0];
    double area = 0.5 * sqrt(n0 * n0 + n1 * n1 + n2 * n2);
    double bary[7][3], w[7];
    quad7(bary, w);
    double r[TRI_REC];
    for (int i = 0; i < TRI_REC; ++i) r[i] = 0.0;
    for (int p = 0; p < 7; ++p) {
        for (int d = 0; d < 3; ++d)
            r[TR_Q + 3 * p + d] = bary[p][0] * v[0][d] + bary[p][1] * v[1][d] + bary[p][2] * v[2][d];
        r[TR_W + p] = w[p] * area;
    }
    for (int a = 0; a < 3; ++a) {
        for (int d = 0; d < 3; ++d) r[TR_P + 3 * a + d] = v[a][d];
        int e = tri_edge[3 * t + a];
        r[TR_C + a] = tri_sign[3 * t + a] * edge_len[e] / (2.0 * area);
    }
    for (int d = 0; d < 3; ++d) r[TR_CEN + d] = __ddiv_rn(__dadd_rn(__dadd_rn(v[0][d], v[1][d]), v[2][d]), 3.0);
    double h = norm3_rn(e1[0], e1[1], e1[2]);
    h = fmax(h, norm3_rn(e2[0], e2[1], e2[2]));
    h = fmax(h, norm3_rn(e3[0], e3[1], e3[2]));
    r[TR_H] = h;
    for (int i = 0; i < TRI_REC; ++i) rec64[t * TRI_REC + i] = r[i];
    // FP32 copy; positions (quadrature points, vertices, centroid) relative to the mesh centre
    const double c[3] = {cx, cy, cz};
    for (int i = 0; i < TRI_REC; ++i) {
        double x = r[i];
        if (i < TR_W) x -= c[(i - TR_Q) % 3];
        else if (i >= TR_P && i < TR_C) x -= c[(i - TR_P) % 3];
        else if (i >= TR_CEN && i < TR_H) x -= c[(i - TR_CEN) % 3];
        rec32[t * TRI_REC + i] = (float)x;
    }
    // centroid as an unevaluated float sum hi + lo, so centroid differences keep FP64-level accuracy
    for (int d = 0; d < 3; ++d) {
        double x = r[TR_CEN + d] - c[d];
        float hi = (float)x;
        rec32[t * TRI_REC + TR_CLO + d] = (float)(x - (double)hi);
    }
}

__device__ inline bool shares_vertex(const int32_t *a, const int32_t *b) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (a[i] == b[j]) return true;
    return false;
}

__device__ inline bool near_pair(const double *rt, const double *rs, const int32_t *vt, const int32_t *vs, double alpha) {
    if (shares_vertex(vt, vs)) return true;
    double dx = __dsub_rn(rt[TR_CEN], rs[TR_CEN]);
    double dy = __dsub_rn(rt[TR_CEN + 1], rs[TR_CEN + 1]);
    double dz = __dsub_rn(rt[TR_CEN + 2], rs[TR_CEN + 2]);
    double h = fmax(rt[TR_H], rs[TR_H]);
    return norm3_rn(dx, dy, dz) < __dmul_rn(alpha, h);
}

// pass 0: count, pass 1: write (t, s) pairs with t <= s
__global__ void k_near(int64_t nt, const double *__restrict__ rec, const int32_t *__restrict__ vid, double alpha,
                       unsigned long long *counter, int32_t *out, int64_t cap) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int64_t t = blockIdx.y; t < nt; t += gridDim.y) {
        if (s >= nt || s < t) continue;
        if (!near_pair(rec + t * TRI_REC, rec + s * TRI_REC, vid + 3 * t, vid + 3 * s, alpha)) continue;
        unsigned long long k = atomicAdd(counter, 1ull);
        if (out && (int64_t)k < cap) {
            out[2 * k] = (int32_t)t;
            out[2 * k + 1] = (int32_t)s;
        }
    }
}

// Sparse RWG Gram rows: [G]_ij = int (n x f_i) . f_j; on triangle t with local
// edges a (row) and b (column) the integrand c_a c_b n.((r-p_a) x (r-p_b)) is
// linear in r, so it integrates exactly to c_a c_b A n.((c-p_a) x (c-p_b)).
__global__ void k_gram_rows(int64_t ne, const double *__restrict__ rec, const int32_t *__restrict__ edge_tri,
                            const int32_t *__restrict__ edge_loc, const int32_t *__restrict__ tri_edge,
                            double *__restrict__ val, int32_t *__restrict__ col) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ne) return;
    for (int s = 0; s < 2; ++s) {
        int t = edge_tri[2 * i + s], a = edge_loc[2 * i + s];
        const double *r = rec + (int64_t)t * TRI_REC;
        // area from weights (sum of weights = area)
        double A = 0;
        for (int p = 0; p < 7; ++p) A += r[TR_W + p];
        const double *pv = r + TR_P;
        double e1[3], e2[3], n[3];
        for (int d = 0; d < 3; ++d) { e1[d] = pv[3 + d] - pv[d]; e2[d] = pv[6 + d] - pv[d]; }
        n[0] = e1[1] * e2[2] - e1[2] * e2[1];
        n[1] = e1[2] * e2[0] - e1[0] * e2[2];
        n[2] = e1[0] * e2[1] - e1[1] * e2[0];
        double nl = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        for (int d = 0; d < 3; ++d) n[d] /= nl;
        double ca[3], cb[3];
        for (int d = 0; d < 3; ++d) ca[d] = r[TR_CEN + d] - pv[3 * a + d];
        for (int b = 0; b < 3; ++b) {
            for (int d = 0; d < 3; ++d) cb[d] = r[TR_CEN + d] - pv[3 * b + d];
            double cr0 = ca[1] * cb[2] - ca[2] * cb[1];
            double cr1 = ca[2] * cb[0] - ca[0] * cb[2];
            double cr2 = ca[0] * cb[1] - ca[1] * cb[0];
            double v = r[TR_C + a] * r[TR_C + b] * A * (n[0] * cr0 + n[1] * cr1 + n[2] * cr2);
            val[6 * i + 3 * s + b] = (b == a) ? 0.0 : v;
            col[6 * i + 3 * s + b] = tri_edge[3 * t + b];
        }
    }
}

__device__ inline void sph_basis(double th, double ph, double rh[3], double thh[3], double phh[3]) {
    double st, ct, sp, cp;
    sincos(th, &st, &ct);
    sincos(ph, &sp, &cp);
    rh[0] = st * cp; rh[1] = st * sp; rh[2] = ct;
    thh[0] = ct * cp; thh[1] = ct * sp; thh[2] = -st;
    phh[0] = -sp; phh[1] = cp; phh[2] = 0.0;
}

// Per wave w: r_hat (arrival direction), polarisation p and k_hat x p
// (k_hat = -r_hat), 9 doubles.
__global__ void k_wave_basis(int nw, const double *__restrict__ waves, double *__restrict__ wb) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nw) return;
    double rh[3], thh[3], phh[3];
    sph_basis(waves[3 * w], waves[3 * w + 1], rh, thh, phh);
    double sps, cps;
    sincos(waves[3 * w + 2], &sps, &cps);
    double p[3];
    for (int d = 0; d < 3; ++d) p[d] = cps * thh[d] + sps * phh[d];
    double *o = wb + 9 * (int64_t)w;
    for (int d = 0; d < 3; ++d) {
        o[d] = rh[d];
        o[3 + d] = p[d];
    }
    o[6] = -(rh[1] * p[2] - rh[2] * p[1]);
    o[7] = -(rh[2] * p[0] - rh[0] * p[2]);
    o[8] = -(rh[0] * p[1] - rh[1] * p[0]);
}

// v^E_i = int f_i . E_inc, v^H_i = -int f_i . H_inc (paper Eq. (v)), one thread
// per (edge, wave); E_inc = p exp(j k0 r_hat . r), H_inc = (k_hat x p)/eta0 (...).
// F32: the integrand in FP32 with the phase factor exp(j k0 r_hat . r) by the
// FP32 reduced sin/cos (the mixed-precision solve), else FP64.
template <bool F32>
__global__ void k_rhs(int64_t ne, int nw, const double *__restrict__ rec, const int32_t *__restrict__ edge_tri,
                      const int32_t *__restrict__ edge_loc, const double *__restrict__ wb, z64 *__restrict__ vE,
                      z64 *__restrict__ vH) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= ne * nw) return;
    int64_t i = idx / nw;
    int w = (int)(idx % nw);
    const double *o = wb + 9 * (int64_t)w;
    const double rh[3] = {o[0], o[1], o[2]}, p[3] = {o[3], o[4], o[5]}, hp[3] = {o[6], o[7], o[8]};
    if constexpr (F32) {   // the whole integrand in FP32 (phase reduced), 14 terms summed in FP32
        const float pf[3] = {(float)p[0], (float)p[1], (float)p[2]},
                    hpf[3] = {(float)(hp[0] / ETA0), (float)(hp[1] / ETA0), (float)(hp[2] / ETA0)};
        float er = 0.f, ei = 0.f, hr = 0.f, hi = 0.f;
        for (int s = 0; s < 2; ++s) {
            const int t = edge_tri[2 * i + s], a = edge_loc[2 * i + s];
            const double *r = rec + (int64_t)t * TRI_REC;
            const float c = (float)r[TR_C + a];
            for (int q = 0; q < 7; ++q) {
                const double *x = r + TR_Q + 3 * q;
                const float f0 = (float)(x[0] - r[TR_P + 3 * a]), f1 = (float)(x[1] - r[TR_P + 3 * a + 1]),
                            f2 = (float)(x[2] - r[TR_P + 3 * a + 2]);
                // the phase argument in FP64 (coordinates may lie far from the origin), reduced in FP32
                const float ph = (float)(K0 * (rh[0] * x[0] + rh[1] * x[1] + rh[2] * x[2]));
                float sn, cs;
                sincos_red(ph, &sn, &cs);
                const float wc = (float)r[TR_W + q] * c;
                const float wfe = wc * (f0 * pf[0] + f1 * pf[1] + f2 * pf[2]);
                const float wfh = -wc * (f0 * hpf[0] + f1 * hpf[1] + f2 * hpf[2]);
                er += wfe * cs; ei += wfe * sn;
                hr += wfh * cs; hi += wfh * sn;
            }
        }
        vE[i * nw + w] = z64(er, ei);
        vH[i * nw + w] = z64(hr, hi);
        return;
    }
    z64 e(0, 0), h(0, 0);
    for (int s = 0; s < 2; ++s) {
        int t = edge_tri[2 * i + s], a = edge_loc[2 * i + s];
        const double *r = rec + (int64_t)t * TRI_REC;
        double c = r[TR_C + a];
        for (int q = 0; q < 7; ++q) {
            const double *x = r + TR_Q + 3 * q;
            double f0 = x[0] - r[TR_P + 3 * a], f1 = x[1] - r[TR_P + 3 * a + 1], f2 = x[2] - r[TR_P + 3 * a + 2];
            double ph = K0 * (rh[0] * x[0] + rh[1] * x[1] + rh[2] * x[2]);
            double sn, cs;
            sincos(ph, &sn, &cs);
            double wfe = r[TR_W + q] * c * (f0 * p[0] + f1 * p[1] + f2 * p[2]);
            double wfh = -r[TR_W + q] * c * (f0 * hp[0] + f1 * hp[1] + f2 * hp[2]) / ETA0;
            e.re += wfe * cs; e.im += wfe * sn;
            h.re += wfh * cs; h.im += wfh * sn;
        }
    }
    vE[i * nw + w] = e;
    vH[i * nw + w] = h;
}

// Far field of J = sum aJ f, M = sum aM f radiating into free space:
// F = (j k0/4pi) [ -eta0 (N - r (r.N)) + r x L ], N = int J e^{j k0 r.r'}, L likewise.
// One block per (rhs, direction); j is (2 ne, nrhs) internal order [M; J].
// F32: each thread's share of the sums in FP32, with the phase factors by the
// FP32 reduced sin/cos (mixed-precision solve); the sums over threads in FP64.
template <bool F32>
__global__ void k_farfield(int64_t nt, int64_t ne, int nrhs, const double *__restrict__ rec,
                           const int32_t *__restrict__ tri_edge, const z64 *__restrict__ j,
                           const double *__restrict__ obs, int ndir, int monostatic,
                           const double *__restrict__ exc, double *__restrict__ rcs) {
    int w = blockIdx.y;
    int dI = blockIdx.x;
    double th, ph;
    if (monostatic) { th = exc[3 * w]; ph = exc[3 * w + 1]; }
    else { th = obs[2 * dI]; ph = obs[2 * dI + 1]; }
    double rh[3], thh[3], phh[3];
    sph_basis(th, ph, rh, thh, phh);
    double acc[12];
    for (int k = 0; k < 12; ++k) acc[k] = 0.0;
    if constexpr (F32) {   // each thread's terms (a few tens) in FP32; the sums over threads below in FP64
        float af[12];
        for (int k = 0; k < 12; ++k) af[k] = 0.f;
        for (int64_t t = threadIdx.x; t < nt; t += blockDim.x) {
            const double *r = rec + t * TRI_REC;
            c32 aJ[3], aM[3];
            for (int a = 0; a < 3; ++a) {
                const int e = tri_edge[3 * t + a];
                const z64 jm = j[(int64_t)e * nrhs + w], jj = j[(ne + e) * nrhs + w];
                const float c = (float)r[TR_C + a];
                aM[a] = c32(c * (float)jm.re, c * (float)jm.im);
                aJ[a] = c32(c * (float)jj.re, c * (float)jj.im);
            }
            for (int q = 0; q < 7; ++q) {
                const double *x = r + TR_Q + 3 * q;
                float sn, cs;
                sincos_red((float)(K0 * (rh[0] * x[0] + rh[1] * x[1] + rh[2] * x[2])), &sn, &cs);
                const float wq = (float)r[TR_W + q];
                const c32 e(cs * wq, sn * wq);
                for (int d = 0; d < 3; ++d) {
                    c32 sJ(0, 0), sM(0, 0);
                    for (int a = 0; a < 3; ++a) {
                        const float f = (float)(x[d] - r[TR_P + 3 * a + d]);
                        sJ += f * aJ[a];
                        sM += f * aM[a];
                    }
                    const c32 vJ = sJ * e, vM = sM * e;
                    af[2 * d] += vJ.re; af[2 * d + 1] += vJ.im;
                    af[6 + 2 * d] += vM.re; af[6 + 2 * d + 1] += vM.im;
                }
            }
        }
        for (int k = 0; k < 12; ++k) acc[k] = af[k];
    } else {
    for (int64_t t = threadIdx.x; t < nt; t += blockDim.x) {
        const double *r = rec + t * TRI_REC;
        z64 aJ[3], aM[3];
        for (int a = 0; a < 3; ++a) {
            int e = tri_edge[3 * t + a];
            aM[a] = r[TR_C + a] * j[(int64_t)e * nrhs + w];
            aJ[a] = r[TR_C + a] * j[(ne + e) * nrhs + w];
        }
        for (int q = 0; q < 7; ++q) {
            const double *x = r + TR_Q + 3 * q;
            double phs = K0 * (rh[0] * x[0] + rh[1] * x[1] + rh[2] * x[2]);
            double sn, cs;
            sincos(phs, &sn, &cs);
            z64 e(cs * r[TR_W + q], sn * r[TR_W + q]);
            for (int d = 0; d < 3; ++d) {
                z64 sJ(0, 0), sM(0, 0);
                for (int a = 0; a < 3; ++a) {
                    double f = x[d] - r[TR_P + 3 * a + d];
                    sJ += f * aJ[a];
                    sM += f * aM[a];
                }
                z64 vJ = sJ * e, vM = sM * e;
                acc[2 * d] += vJ.re; acc[2 * d + 1] += vJ.im;
                acc[6 + 2 * d] += vM.re; acc[6 + 2 * d + 1] += vM.im;
            }
        }
    }
    }
    __shared__ double red[12][32];
    for (int k = 0; k < 12; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int nwarp = blockDim.x >> 5;
        double s[12];
        for (int k = 0; k < 12; ++k) {
            s[k] = 0;
            for (int i = 0; i < nwarp; ++i) s[k] += red[k][i];
        }
        z64 N[3], L[3];
        for (int d = 0; d < 3; ++d) { N[d] = z64(s[2 * d], s[2 * d + 1]); L[d] = z64(s[6 + 2 * d], s[6 + 2 * d + 1]); }
        z64 Nth = thh[0] * N[0] + thh[1] * N[1] + thh[2] * N[2];
        z64 Nph = phh[0] * N[0] + phh[1] * N[1] + phh[2] * N[2];
        z64 Lth = thh[0] * L[0] + thh[1] * L[1] + thh[2] * L[2];
        z64 Lph = phh[0] * L[0] + phh[1] * L[1] + phh[2] * L[2];
        // F = (j k0 / 4 pi) (-eta0 N_perp + r x L), r x L = L_th phi - L_ph theta
        z64 Fth = -ETA0 * Nth - Lph;
        z64 Fph = -ETA0 * Nph + Lth;
        double pre = K0 / (4.0 * PI);
        int nd = monostatic ? 1 : ndir;
        rcs[((int64_t)w * nd + dI) * 2 + 0] = 4.0 * PI * pre * pre * norm2(Fth);
        rcs[((int64_t)w * nd + dI) * 2 + 1] = 4.0 * PI * pre * pre * norm2(Fph);
    }
}

}  // namespace

void launch_tri_records(Mesh &m, const double *d_verts, const int32_t *d_tris, cudaStream_t st) {
    int64_t nt = m.h.nt;
    DevBuf<int32_t> d_sign;
    DevBuf<double> d_len;
    d_sign.alloc(3 * nt);
    d_len.alloc(m.h.ne);
    CBFM_CUDA(cudaMemcpyAsync(d_sign.p, m.h.tri_sign.data(), 3 * nt * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CBFM_CUDA(cudaMemcpyAsync(d_len.p, m.h.edge_len.data(), m.h.ne * sizeof(double), cudaMemcpyHostToDevice, st));
    {
        ProfScope ps_("k_tri_records", st);
        k_tri_records<<<(unsigned)((nt + 127) / 128), 128, 0, st>>>(nt, d_verts, d_tris, m.tri_edge.p, d_sign.p, d_len.p,
                                                                    m.centre[0], m.centre[1], m.centre[2], m.tri64.p,
                                                                    m.tri32.p);
        launched("k_tri_records");
    }
    CBFM_CUDA(cudaStreamSynchronize(st));
}

void launch_near_pairs(Mesh &m, cudaStream_t st) {
    int64_t nt = m.h.nt;
    DevBuf<unsigned long long> cnt;
    cnt.alloc(1);
    CBFM_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long), st));
    dim3 grid((unsigned)((nt + 255) / 256), (unsigned)(nt < 65535 ? nt : 65535));
    {
        ProfScope ps_("k_near(count)", st);
        k_near<<<grid, 256, 0, st>>>(nt, m.tri64.p, m.tri_vid.p, m.alpha, cnt.p, nullptr, 0);
        launched("k_near(count)");
    }
    unsigned long long n = 0;
    CBFM_CUDA(cudaMemcpyAsync(&n, cnt.p, sizeof(n), cudaMemcpyDeviceToHost, st));
    CBFM_CUDA(cudaStreamSynchronize(st));
    m.n_near = (int64_t)n;
    m.near_pairs.alloc(2 * n);
    CBFM_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long), st));
    {
        ProfScope ps_("k_near(fill)", st);
        k_near<<<grid, 256, 0, st>>>(nt, m.tri64.p, m.tri_vid.p, m.alpha, cnt.p, m.near_pairs.p, (int64_t)n);
        launched("k_near(fill)");
    }
}

void launch_gram_rows(Mesh &m, cudaStream_t st) {
    int64_t ne = m.h.ne;
    m.gram_val.alloc(6 * ne);
    m.gram_col.alloc(6 * ne);
    {
        ProfScope ps_("k_gram_rows", st);
        k_gram_rows<<<(unsigned)((ne + 127) / 128), 128, 0, st>>>(ne, m.tri64.p, m.edge_tri.p, m.edge_loc.p, m.tri_edge.p,
                                                                  m.gram_val.p, m.gram_col.p);
        launched("k_gram_rows");
    }
}

void launch_rhs(const Mesh &m, const double *d_waves, int nw, z64 *vE, z64 *vH, cudaStream_t st, bool f32) {
    int64_t tot = m.h.ne * (int64_t)nw;
    DevBuf<double> wb;
    wb.alloc((size_t)9 * nw);
    k_wave_basis<<<(unsigned)((nw + 127) / 128), 128, 0, st>>>(nw, d_waves, wb.p);
    launched("k_wave_basis");
    {
        ProfScope ps_("k_rhs", st);
        const unsigned g = (unsigned)((tot + 127) / 128);
        if (f32) k_rhs<true><<<g, 128, 0, st>>>(m.h.ne, nw, m.tri64.p, m.edge_tri.p, m.edge_loc.p, wb.p, vE, vH);
        else k_rhs<false><<<g, 128, 0, st>>>(m.h.ne, nw, m.tri64.p, m.edge_tri.p, m.edge_loc.p, wb.p, vE, vH);
        launched("k_rhs");
    }
}

void launch_farfield(const Mesh &m, const z64 *j, int nrhs, const double *d_obs, int ndir, bool monostatic,
                     const double *d_exc, double *d_rcs, cudaStream_t st, bool f32) {
    dim3 grid(monostatic ? 1 : ndir, nrhs);
    {
        ProfScope ps_("k_farfield", st);
        if (f32)
            k_farfield<true><<<grid, 256, 0, st>>>(m.h.nt, m.h.ne, nrhs, m.tri64.p, m.tri_edge.p, j, d_obs, ndir,
                                                   monostatic ? 1 : 0, d_exc, d_rcs);
        else
            k_farfield<false><<<grid, 256, 0, st>>>(m.h.nt, m.h.ne, nrhs, m.tri64.p, m.tri_edge.p, j, d_obs, ndir,
                                                    monostatic ? 1 : 0, d_exc, d_rcs);
        launched("k_farfield");
    }
}

}  // namespace cbfm
