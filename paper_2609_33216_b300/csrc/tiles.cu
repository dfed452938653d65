// Kernel-entry tile generator: blocks of the symmetric Muller-like matrix
// (Eq. 15; unscaled baseline of Sec. 6), or of the PMCHWT (Eq. symmetric_pmchwt) or
// Burton-Miller (Eq. bm) comparators, between two point lists.
//
// Each thread owns one point of the "thread" list; a chunk of the "loop" list is
// staged in shared memory.  For every (thread point, loop point) pair the thread
// evaluates H_0 and H_1 at k0 r and k1 r once and produces the whole 2x2 block
// [A11 A12; A21 A22] of the pair, writing the entries whose slots are present.
// Consecutive threads own consecutive output rows, so stores are coalesced.
//
// Kernel forms (d = x_obs - x_src, r = |d|, a = d.nu_obs, b = d.nu_src):
//   G    = (i/4) H0(kr)
//   D    = (ik/4) H1(kr) b/r          (normal derivative in the source, Sec. 3.1)
//   D*   = -(ik/4) H1(kr) a/r         (normal derivative in the observation point)
//   N    = (ik/4) [H1(kr) nu_o.nu_s / r + (ab/r)(k H0(kr)/r - 2 H1(kr)/r^2)]
// Swapping the two points negates d exactly, so a' = -b and b' = -a exactly and r,
// ab and nu_o.nu_s are unchanged; with the explicit round-to-nearest intrinsics
// below, A12(p,q) and A21(q,p) go through identical operations and the matrix is
// symmetric bit for bit away from the diagonal (Eq. syms).
//
// The one-point corrected diagonal (Sec. 3.1) applies when both points carry the
// same node id:
//   S~_k   = i/4 - (gamma_E + log(k w / 4 pi)) / (2 pi)
//   D~ = D*~ = -kappa / (4 pi)
//   (N_k0 - N_k1)~ = (i/8)(k0^2 - k1^2) - [k0^2 (log(k0/2) + gamma_E) - k1^2 (log(k1/2) + gamma_E)] / (4 pi)
//                    + (k0^2 - k1^2) / (8 pi) - (k0^2 - k1^2) log(w / 2 pi) / (4 pi)
//   PMCHWT: N~_k = (hs - pi/6) / w^2 + kappa^2 / (24 pi) + (the k-dependent terms above for one k):
//   the zeta-corrected trapezoidal weight of the 1/tau^2 singularity, -2 zeta(2)/h, on the
//   Laplace part 1/(2 pi |gamma'| tau^2) in the parameter tau, plus the constant term of the
//   kernel times the source speed: kappa^2/(24 pi) and the speed term hs / w^2 (zero on a
//   circle; hs from the node weights, see speed_terms).
// H_0 and H_1 come from hankel01() (hankel.cuh), accurate to about 1e-15 at every
// argument.
#include "common.cuh"
#include "hankel.cuh"

namespace symhss {

namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kEulerGamma = 0.577215664901532860606512090082402431;

struct LayerVals { double2 g, d, ds, n; };

// S, D, D*, N kernels of one wavenumber at a non-coincident pair; lr = log(r),
// inv_r = 1/r, lhk = log(k/2), ik = 1/k.
__device__ __forceinline__ LayerVals layer(double k, double r, double inv_r, double lr, double lhk, double ik,
                                           double a_r, double b_r, double nn_r, double ab_r) {
  const double z = __dmul_rn(k, r);
  double2 h0, h1;
  hankel01(z, lr + lhk, inv_r * ik, h0, h1);
  const double j0v = h0.x, y0v = h0.y, j1v = h1.x, y1v = h1.y;
  const double kq = 0.25 * k;
  LayerVals v;
  v.g = make_double2(-0.25 * y0v, 0.25 * j0v);
  const double2 c1 = make_double2(-__dmul_rn(kq, y1v), __dmul_rn(kq, j1v));
  v.d = make_double2(__dmul_rn(c1.x, b_r), __dmul_rn(c1.y, b_r));
  v.ds = make_double2(-__dmul_rn(c1.x, a_r), -__dmul_rn(c1.y, a_r));
  // N = c1 * nn/r + i kq (ab/r) (k H0 / r - 2 H1 / r^2)
  const double2 qv = make_double2(k * j0v * inv_r - 2.0 * j1v * inv_r * inv_r,
                                  k * y0v * inv_r - 2.0 * y1v * inv_r * inv_r);
  const double s = kq * ab_r;
  v.n = make_double2(c1.x * nn_r - s * qv.y, c1.y * nn_r + s * qv.x);
  return v;
}

// e_a * u - e_b * v, component-wise, without contraction
__device__ __forceinline__ double2 combo(double ea, double2 u, double eb, double2 v) {
  return make_double2(__dsub_rn(__dmul_rn(ea, u.x), __dmul_rn(eb, v.x)),
                      __dsub_rn(__dmul_rn(ea, u.y), __dmul_rn(eb, v.y)));
}
__device__ __forceinline__ double2 rscale(double s, double2 u) {
  return make_double2(__dmul_rn(s, u.x), __dmul_rn(s, u.y));
}

struct P7 { double x, y, nx, ny, w, kappa, hs; int id; };

// 2x2 block [A11 A12; A21 A22] for observation o, source s.
__device__ __forceinline__ void pair_block(const P7& o, const P7& s, const KernelParams& kp,
                                           bool unscaled, double2 out[4]) {
  const double wgt = unscaled ? s.w : __dmul_rn(o.w, s.w);
  if (o.id >= 0 && o.id == s.id && kp.form == SYMHSS_BM) {
    // Burton-Miller: [-e0 S0 - a e0 (D*0 + I/2), D0 - I/2 + a N0; -e1 S1, D1 + I/2], a = i/k0
    const double w = o.w;
    const double c = 1.0 / (2.0 * kPi);
    const double2 gs0 = make_double2(-c * (kEulerGamma + log(kp.k0 * w / (4.0 * kPi))), 0.25);
    const double2 gs1 = make_double2(-c * (kEulerGamma + log(kp.k1 * w / (4.0 * kPi))), 0.25);
    const double dd = -o.kappa / (4.0 * kPi);
    const double lw = log(w / (2.0 * kPi));
    const double k0s = kp.k0 * kp.k0;
    const double hyp = (o.hs - kPi / 6.0) / (w * w) + o.kappa * o.kappa / (24.0 * kPi);
    const double2 n0 = make_double2(hyp - k0s * (kp.lhk0 + kEulerGamma) / (4.0 * kPi) + k0s / (8.0 * kPi) -
                                        k0s / (4.0 * kPi) * lw,
                                    0.125 * k0s);
    const double ae = kp.eps0 * kp.ik0;  // |a| eps0
    const double ft = unscaled ? 1.0 : w;
    // -e0 S0 - i ae D*0, then - i ae / 2 (free term)
    out[0] = make_double2(wgt * (-kp.eps0 * gs0.x), wgt * (-kp.eps0 * gs0.y - ae * dd) - 0.5 * ae * ft);
    // D0 + i (1/k0) N0 - 1/2
    out[1] = make_double2(wgt * (dd - kp.ik0 * n0.y) - 0.5 * ft, wgt * (kp.ik0 * n0.x));
    out[2] = make_double2(wgt * (-kp.eps1 * gs1.x), wgt * (-kp.eps1 * gs1.y));
    out[3] = make_double2(wgt * dd + 0.5 * ft, 0.0);
    return;
  }
  if (o.id >= 0 && o.id == s.id) {
    const double w = o.w;
    const double c = 1.0 / (2.0 * kPi);
    const double2 gs0 = make_double2(-c * (kEulerGamma + log(kp.k0 * w / (4.0 * kPi))), 0.25);
    const double2 gs1 = make_double2(-c * (kEulerGamma + log(kp.k1 * w / (4.0 * kPi))), 0.25);
    const double2 ks = combo(kp.cs0, gs0, kp.cs1, gs1);
    const double dd = -o.kappa / (4.0 * kPi);
    const double kd = kp.cd0 * dd - kp.cd1 * dd;
    // k-dependent part of N~_k: (i/8) k^2 - k^2 (log(k/2) + gamma_E)/(4 pi) + k^2/(8 pi)
    //                           - k^2 log(w / 2 pi)/(4 pi)
    const double lw = log(w / (2.0 * kPi));
    const double k0s = kp.k0 * kp.k0, k1s = kp.k1 * kp.k1;
    const double f0 = -k0s * (kp.lhk0 + kEulerGamma) / (4.0 * kPi) + k0s / (8.0 * kPi) - k0s / (4.0 * kPi) * lw;
    const double f1 = -k1s * (kp.lhk1 + kEulerGamma) / (4.0 * kPi) + k1s / (8.0 * kPi) - k1s / (4.0 * kPi) * lw;
    double2 kn;
    if (kp.form == SYMHSS_PMCHWT) {
      // hypersingular part: -pi / (6 w^2) (zeta-corrected 1/tau^2) + kappa^2 / (24 pi) + hs / w^2
      const double hyp = (o.hs - kPi / 6.0) / (w * w) + o.kappa * o.kappa / (24.0 * kPi);
      kn = make_double2(kp.cn0 * (hyp + f0) - kp.cn1 * (hyp + f1), 0.125 * (kp.cn0 * k0s - kp.cn1 * k1s));
    } else {
      // the hypersingular parts cancel in N_k0 - N_k1
      const double dk2 = k0s - k1s;
      const double nre = -(k0s * (kp.lhk0 + kEulerGamma) - k1s * (kp.lhk1 + kEulerGamma)) / (4.0 * kPi) +
                         dk2 / (8.0 * kPi) - dk2 / (4.0 * kPi) * lw;
      kn = make_double2(nre, 0.125 * dk2);
      (void)f0; (void)f1;
    }
    const double ft = kp.half_ft * (unscaled ? 1.0 : w);
    out[0] = make_double2(-wgt * ks.x, -wgt * ks.y);
    out[1] = make_double2(wgt * kd - ft, 0.0);
    out[2] = make_double2(wgt * kd + ft, 0.0);
    out[3] = make_double2(-wgt * kn.x, -wgt * kn.y);
    return;
  }
  const double dx = __dsub_rn(o.x, s.x), dy = __dsub_rn(o.y, s.y);
  const double r = __dsqrt_rn(__fma_rn(dx, dx, __dmul_rn(dy, dy)));
  const double a = __fma_rn(dx, o.nx, __dmul_rn(dy, o.ny));
  const double b = __fma_rn(dx, s.nx, __dmul_rn(dy, s.ny));
  const double nn = __fma_rn(o.nx, s.nx, __dmul_rn(o.ny, s.ny));
  // one reciprocal and one logarithm per pair; products with inv_r keep the exact
  // sign symmetry of the quotients under the swap of the two points
  const double inv_r = __drcp_rn(r);
  const double lr = log(r);
  const double a_r = __dmul_rn(a, inv_r), b_r = __dmul_rn(b, inv_r);
  const double nn_r = __dmul_rn(nn, inv_r), ab_r = __dmul_rn(__dmul_rn(a, b), inv_r);
  const LayerVals l0 = layer(kp.k0, r, inv_r, lr, kp.lhk0, kp.ik0, a_r, b_r, nn_r, ab_r);
  const LayerVals l1 = layer(kp.k1, r, inv_r, lr, kp.lhk1, kp.ik1, a_r, b_r, nn_r, ab_r);
  if (kp.form == SYMHSS_BM) {
    const double ae = kp.eps0 * kp.ik0;
    // -e0 G0 - i ae D*0 ;  D0 + i (1/k0) N0 ;  -e1 G1 ;  D1
    out[0] = rscale(wgt, make_double2(-kp.eps0 * l0.g.x + ae * l0.ds.y, -kp.eps0 * l0.g.y - ae * l0.ds.x));
    out[1] = rscale(wgt, make_double2(l0.d.x - kp.ik0 * l0.n.y, l0.d.y + kp.ik0 * l0.n.x));
    out[2] = rscale(wgt, make_double2(-kp.eps1 * l1.g.x, -kp.eps1 * l1.g.y));
    out[3] = rscale(wgt, l1.d);
    return;
  }
  const double2 ks = combo(kp.cs0, l0.g, kp.cs1, l1.g);
  const double2 kd = combo(kp.cd0, l0.d, kp.cd1, l1.d);
  const double2 kds = combo(kp.cd0, l0.ds, kp.cd1, l1.ds);
  const double2 kn = combo(kp.cn0, l0.n, kp.cn1, l1.n);
  const double2 t11 = rscale(wgt, ks), t22 = rscale(wgt, kn);
  out[0] = make_double2(-t11.x, -t11.y);
  out[1] = rscale(wgt, kd);
  out[2] = rscale(wgt, kds);
  out[3] = make_double2(-t22.x, -t22.y);
}

__global__ void __launch_bounds__(TILE_T) tile_kernel(const TileLaunch a) {
  __shared__ double sx[TILE_L], sy[TILE_L], snx[TILE_L], sny[TILE_L], sw[TILE_L], sk[TILE_L], shs[TILE_L];
  __shared__ int sid[TILE_L], ss0[TILE_L], ss1[TILE_L];
  const TileChunk ch = a.chunks[blockIdx.x];
  const TileJob jb = a.jobs[ch.job];
  const int nl = min(min(TILE_L, ch.ln), jb.n_lp - ch.l0);
  const int t = threadIdx.x;
  if (t < nl) {
    const int li = jb.lp_off + ch.l0 + t;
    const int p = a.lp_pt[li];
    sx[t] = a.lpts.x[p]; sy[t] = a.lpts.y[p]; snx[t] = a.lpts.nx[p]; sny[t] = a.lpts.ny[p];
    sw[t] = a.lpts.w[p]; sk[t] = a.lpts.kappa[p]; sid[t] = a.lpts.id[p];
    shs[t] = a.lpts.hs ? a.lpts.hs[p] : 0.0;
    ss0[t] = a.lp_s0[li]; ss1[t] = a.lp_s1[li];
  }
  __syncthreads();
  const int ti = ch.t0 + t;
  if (ti >= jb.n_tp) return;
  const int tidx = jb.tp_off + ti;
  const int p = a.tp_pt[tidx];
  P7 tp;
  tp.x = a.tpts.x[p]; tp.y = a.tpts.y[p]; tp.nx = a.tpts.nx[p]; tp.ny = a.tpts.ny[p];
  tp.w = a.tpts.w[p]; tp.kappa = a.tpts.kappa[p]; tp.id = a.tpts.id[p];
  tp.hs = a.tpts.hs ? a.tpts.hs[p] : 0.0;
  const int ts0 = a.tp_s0[tidx], ts1 = a.tp_s1[tidx];
  const bool src_thread = (jb.flags & TILE_SRC_IS_THREAD) != 0;
  const bool unscaled = (jb.flags & TILE_UNSCALED) != 0;
  const KernelParams kp = a.kps[jb.prm];
  if (ts0 >= jb.ld || ts1 >= jb.ld) { atomicOr(a.status, ST_BAD_INDEX); return; }
  double2* out = a.out + jb.out_off;
  const bool symd = (jb.flags & TILE_SYM_DIAG) != 0 && !src_thread;
  for (int l = 0; l < nl; ++l) {
    if (symd && ch.l0 + l < ti) continue;  // the pair (j, i) of j < i is written by thread j
    P7 lp;
    lp.x = sx[l]; lp.y = sy[l]; lp.nx = snx[l]; lp.ny = sny[l]; lp.w = sw[l]; lp.kappa = sk[l]; lp.hs = shs[l];
    lp.id = sid[l];
    const int ls0 = ss0[l], ls1 = ss1[l];
    if ((ts0 < 0 && ts1 < 0) || (ls0 < 0 && ls1 < 0)) continue;
    double2 blk[4];
    if (src_thread) pair_block(lp, tp, kp, unscaled, blk);
    else pair_block(tp, lp, kp, unscaled, blk);
    // blk[e*2 + c]; thread slots are equations (normal) or unknowns (transposed)
    const int tsl[2] = {ts0, ts1};
    const int lsl[2] = {ls0, ls1};
#pragma unroll
    for (int e = 0; e < 2; ++e) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int row = src_thread ? tsl[c] : tsl[e];
        const int col = src_thread ? lsl[e] : lsl[c];
        if (row >= 0 && col >= 0) out[row + (long long)col * jb.ld] = blk[e * 2 + c];
      }
    }
    if (symd && ch.l0 + l != ti) {
      // the transposed position of every entry (the pair (j, i))
#pragma unroll
      for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int c = 0; c < 2; ++c)
          if (tsl[e] >= 0 && lsl[c] >= 0) out[lsl[c] + (long long)tsl[e] * jb.ld] = blk[e * 2 + c];
    }
  }
}

__global__ void hankel_kernel(const double* x, int n, double2* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double2 h0, h1;
  hankel01(x[i], h0, h1);
  out[i] = h0;
  out[n + i] = h1;
}

}  // namespace

cudaError_t launch_hankel(const double* x, int n, double2* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  hankel_kernel<<<(n + 127) / 128, 128, 0, s>>>(x, n, out);
  symhss::count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_tiles(const TileLaunch& a, cudaStream_t s) {
  if (a.nchunks <= 0) return cudaSuccess;
  tile_kernel<<<a.nchunks, TILE_T, 0, s>>>(a);
  symhss::count_launches(1);
  return cudaGetLastError();
}

}  // namespace symhss
