// The paper's optimisation procedure (arXiv 2207.06374, Sec. "Optimization
// procedure"; Algorithm "TRSTMI optimization steps", steps 2 and 3): for each
// smoothing parameter delta_k in turn, trust-region iterations on the smooth
// maximum F_{s,delta_k} of the variable V, each step from CG-Steihaug
// (Algorithm "Trust-Region CG-Steihaug", after Nocedal and Wright Alg. 7.2),
// the previous stage's result starting the next; repeated from L random
// initialisations, the minimum over the trials returned.
//
// L frames advance together: every objective evaluation is one smooth-maximum
// pass over the stack of frames (lse.cu, a smoothing parameter per frame),
// every vector update one launch over all frames with a coefficient per frame,
// every inner product one launch with a CTA per frame (a fixed reduction
// order).  The host keeps each frame's scalars and runs the algorithms' scalar
// logic per frame; a frame that is not stepping gets zero coefficients, so its
// vectors do not change.  Each frame therefore follows exactly the trajectory
// it follows alone (L = 1).  The model's B is the Hessian of F at the iterate
// (the paper's B_k = grad^2 f_k): its products are formed exactly by the
// chain rule through the column normalisation, the Gram entries and the
// softmax weights (hessian = 0), or, as a diagnosis option, by central
// differences of the exact gradient (hessian = 1); all in binary64.
//
// Per trust-region iteration (Nocedal and Wright Alg. 4.1): g = grad F; the
// stage ends when |g| <= gtol; p from CG-Steihaug with eps = min(1/2,
// sqrt|g|)|g|; rho = (F(V) - F(V + p)) / (-m(p)); radius / 4 if rho < 1/4,
// doubled (capped) if rho > 3/4 and |p| reached it; accept if rho > eta, then
// every column of V is divided by its norm (F is unchanged by that); the stage
// also ends after max_outer iterations or when the radius falls below 1e-14.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "kernels.h"

namespace trstmi {

namespace {

constexpr int kDotThreads = 1024;
constexpr int kCoefRing = 32;     // coefficient buffers in flight between two syncs

// frame f: out = a[f] x + b[f] y over its n entries
__global__ void k_axpby(long long n, long long total, const double* a, const double* x,
                        const double* b, const double* y, double* out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= total) return;
  const long long f = i / n;
  out[i] = a[f] * x[i] + b[f] * y[i];
}

// frame f = blockIdx.x: out[3f] = x.y, out[3f+1] = x.z, out[3f+2] = z.z (z may be
// null): each thread's strided partial, then a fixed tree
__global__ void __launch_bounds__(kDotThreads) k_dots(long long n, const double* x,
                                                      const double* y, const double* z,
                                                      double* out) {
  __shared__ double red[3][kDotThreads];
  const long long base = blockIdx.x * n;
  double a = 0.0, b = 0.0, c = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    a += x[base + i] * y[base + i];
    if (z) { b += x[base + i] * z[base + i]; c += z[base + i] * z[base + i]; }
  }
  red[0][threadIdx.x] = a; red[1][threadIdx.x] = b; red[2][threadIdx.x] = c;
  __syncthreads();
  for (int s = kDotThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      red[0][threadIdx.x] += red[0][threadIdx.x + s];
      red[1][threadIdx.x] += red[1][threadIdx.x + s];
      red[2][threadIdx.x] += red[2][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[3 * blockIdx.x] = red[0][0];
    out[3 * blockIdx.x + 1] = red[1][0];
    out[3 * blockIdx.x + 2] = red[2][0];
  }
}

// frame f = blockIdx.x: the five products of a CG-Steihaug step, in the same
// order of operations as k_dots: out[5f..5f+4] = d.Bd, d.r, p.p, p.d, d.d
__global__ void __launch_bounds__(kDotThreads) k_dots5(long long n, const double* dv,
                                                       const double* bd, const double* r,
                                                       const double* p, double* out) {
  __shared__ double red[5][kDotThreads];
  const long long base = blockIdx.x * n;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0, a4 = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    const double x = dv[base + i], pi = p[base + i];
    a0 += x * bd[base + i];
    a1 += x * r[base + i];
    a2 += pi * pi;
    a3 += pi * x;
    a4 += x * x;
  }
  red[0][threadIdx.x] = a0; red[1][threadIdx.x] = a1; red[2][threadIdx.x] = a2;
  red[3][threadIdx.x] = a3; red[4][threadIdx.x] = a4;
  __syncthreads();
  for (int s = kDotThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < 5; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 5) out[5 * blockIdx.x + threadIdx.x] = red[threadIdx.x][0];
}

// the coefficients of a Hessian product from nu^2 = u.u (dots[3f]): the step
// h / nu along u, and nu / 2h for the difference (zeros when u = 0).  Layout of
// c: [1 ...][step ...][-step ...][nu/2h ...][-nu/2h ...], L each.
__global__ void k_hv_coef(int L, const double* dots, double h, double* c) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= L) return;
  const double nu = sqrt(dots[3 * f]);
  const double step = nu > 0.0 ? h / nu : 0.0, q = nu > 0.0 ? nu / (2.0 * h) : 0.0;
  c[f] = 1.0;
  c[L + f] = step;
  c[2 * L + f] = -step;
  c[3 * L + f] = q;
  c[4 * L + f] = -q;
}

// where flag[f]: frame f's columns divided by their norms (a zero column sets bad[f])
__global__ void k_unit_columns(int N, int d, int L, double2* v, const int* flag, uint32_t* bad) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= (long long)L * N) return;
  const int f = (int)(g / N);
  if (flag && !flag[f]) return;
  double2* col = v + g * d;
  double s = 0.0;
  for (int i = 0; i < d; ++i) s += col[i].x * col[i].x + col[i].y * col[i].y;
  if (!(s > 0.0)) { bad[f] = 1u; return; }
  const double r = sqrt(s);
  for (int i = 0; i < d; ++i) col[i] = make_double2(col[i].x / r, col[i].y / r);
}

// where flag[f]: frame f of dst = frame f of src
__global__ void k_copy_frames(long long n, long long total, const int* flag, const double* src,
                              double* dst) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= total || !flag[i / n]) return;
  dst[i] = src[i];
}

// ---------------------------------------------- exact Hessian products (stack)
// B u for every frame, by differentiating the gradient of F along u:
//   phi_k = v_k / r_k,  d phi_k = (u_k - phi_k Re(phi_k^* u_k)) / r_k,
//   d r_k = Re(phi_k^* u_k),  dG_jk = d phi_j^* phi_k + phi_j^* d phi_k,
//   dx_jk = 2 Re(conj(G_jk) dG_jk),  w = e / S with e = exp((x - s)/delta),
//   dw_jk = w_jk (dx_jk - T) / delta, T = sum w dx (the shift s cancels),
//   dM_jk = dw_jk G_jk + w_jk dG_jk,  g_k = 2 sum_{j != k} M_jk phi_j (M
//   Hermitian), dg_k = 2 sum_{j != k} (dM_jk phi_j + M_jk d phi_j),
//   rho_k = Re(phi_k^* g_k),  d rho_k = Re(d phi_k^* g_k + phi_k^* dg_k),
//   (B u)_k = (dg_k - d phi_k rho_k - phi_k d rho_k) / r_k - grad_k d r_k / r_k
// with grad_k = (g_k - phi_k rho_k) / r_k.  Per pair the passes keep G, dG,
// x (then e) and dx; every sum runs in a fixed order.

constexpr int kHvBlocks = 64;       // CTAs per frame of the weight pass
constexpr int kHvPair = 6;          // doubles per pair: G (2), dG (2), x -> e, dx

// unit columns phi, d phi, r and Re(phi^* u) of every (frame, column)
__global__ void k_hvx_cols(int N, int d, int L, const double2* x, const double2* u, double2* phi,
                           double2* dphi, double* r_out, double* pu_out) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= (long long)L * N) return;
  const double2* xc = x + g * d;
  const double2* uc = u + g * d;
  double q = 0.0;
  for (int i = 0; i < d; ++i) q = fma(xc[i].y, xc[i].y, fma(xc[i].x, xc[i].x, q));
  const double r = sqrt(q), inv = 1.0 / r;
  double pu = 0.0;
  for (int i = 0; i < d; ++i) {
    const double2 ph = make_double2(xc[i].x * inv, xc[i].y * inv);
    phi[g * d + i] = ph;
    pu = fma(ph.y, uc[i].y, fma(ph.x, uc[i].x, pu));
  }
  for (int i = 0; i < d; ++i) {
    const double2 ph = phi[g * d + i];
    dphi[g * d + i] = make_double2((uc[i].x - ph.x * pu) * inv, (uc[i].y - ph.y * pu) * inv);
  }
  r_out[g] = r;
  pu_out[g] = pu;
}

// pair (j, k), j = blockIdx.x < k, of frame blockIdx.y: G, dG, x = |G|^2,
// dx; the frame's max of x (exact, so the order of the atomics is immaterial)
__global__ void k_hvx_pairs(int N, int d, long long P, const double2* phi, const double2* dphi,
                            double* pr, unsigned long long* smax_bits) {
  const int f = blockIdx.y, j = blockIdx.x;
  const double2* ph = phi + (size_t)f * N * d;
  const double2* dp = dphi + (size_t)f * N * d;
  double* out = pr + (size_t)f * P * kHvPair;
  double hi_x = 0.0;
  const long long base = (long long)j * N - (long long)j * (j + 1) / 2 - j - 1;
  for (int k = j + 1 + threadIdx.x; k < N; k += blockDim.x) {
    double gr = 0.0, gi = 0.0, hr = 0.0, hi = 0.0;
    for (int i = 0; i < d; ++i) {
      const double2 a = ph[(size_t)j * d + i], c = ph[(size_t)k * d + i];
      const double2 da = dp[(size_t)j * d + i], dc = dp[(size_t)k * d + i];
      gr = fma(a.x, c.x, gr); gr = fma(a.y, c.y, gr);
      gi = fma(a.x, c.y, gi); gi = fma(-a.y, c.x, gi);
      hr = fma(da.x, c.x, hr); hr = fma(da.y, c.y, hr); hr = fma(a.x, dc.x, hr); hr = fma(a.y, dc.y, hr);
      hi = fma(da.x, c.y, hi); hi = fma(-da.y, c.x, hi); hi = fma(a.x, dc.y, hi); hi = fma(-a.y, dc.x, hi);
    }
    const double x = gr * gr + gi * gi, dx = 2.0 * (gr * hr + gi * hi);
    double* o = out + (size_t)(base + k) * kHvPair;
    o[0] = gr; o[1] = gi; o[2] = hr; o[3] = hi; o[4] = x; o[5] = dx;
    hi_x = fmax(hi_x, x);
  }
  for (int m = 16; m > 0; m >>= 1) hi_x = fmax(hi_x, __shfl_xor_sync(0xffffffffu, hi_x, m));
  if ((threadIdx.x & 31) == 0) atomicMax(smax_bits + f, (unsigned long long)__double_as_longlong(hi_x));
}

// e = exp((x - s)/delta) in place of x; per CTA the partial sums of e and of
// e dx (thread-strided, then a fixed tree) into part[(f * kHvBlocks + b) * 2]
__global__ void __launch_bounds__(256) k_hvx_weights(long long P, const double* deltas,
                                                     const unsigned long long* smax_bits,
                                                     double* pr, double* part) {
  __shared__ double red[2][256];
  const int f = blockIdx.y, b = blockIdx.x;
  double* fp = pr + (size_t)f * P * kHvPair;
  const double s = __longlong_as_double((long long)smax_bits[f]);
  const double inv_delta = 1.0 / deltas[f];
  double se = 0.0, sd = 0.0;
  for (long long q = (long long)b * blockDim.x + threadIdx.x; q < P; q += (long long)kHvBlocks * blockDim.x) {
    double* o = fp + (size_t)q * kHvPair;
    const double e = exp((o[4] - s) * inv_delta);
    o[4] = e;
    se += e;
    sd = fma(e, o[5], sd);
  }
  red[0][threadIdx.x] = se;
  red[1][threadIdx.x] = sd;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      red[0][threadIdx.x] += red[0][threadIdx.x + st];
      red[1][threadIdx.x] += red[1][threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[((size_t)f * kHvBlocks + b) * 2] = red[0][0];
    part[((size_t)f * kHvBlocks + b) * 2 + 1] = red[1][0];
  }
}

// per frame: S = sum e and T = (sum e dx) / S over the CTAs, in order
__global__ void k_hvx_totals(int L, const double* part, double* ST) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= L) return;
  double S = 0.0, Td = 0.0;
  for (int b = 0; b < kHvBlocks; ++b) {
    S += part[((size_t)f * kHvBlocks + b) * 2];
    Td += part[((size_t)f * kHvBlocks + b) * 2 + 1];
  }
  ST[2 * f] = S;
  ST[2 * f + 1] = Td / S;
}

// M = w G in place of G, dM = dw G + w dG in place of dG
__global__ void k_hvx_dm(long long P, int L, const double* deltas, const double* ST, double* pr) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= (long long)L * P) return;
  const int f = (int)(g / P);
  double* o = pr + (size_t)g * kHvPair;
  const double w = o[4] / ST[2 * f];
  const double dw = w * (o[5] - ST[2 * f + 1]) / deltas[f];
  const double gr = o[0], gi = o[1];
  o[2] = fma(dw, gr, w * o[2]);
  o[3] = fma(dw, gi, w * o[3]);
  o[0] = w * gr;
  o[1] = w * gi;
}

// column k = blockIdx.x of frame blockIdx.y, entry i = threadIdx.x (< d):
// g_k and dg_k over j ascending, then rho, d rho (fixed tree over the
// entries) and (B u)_k
__global__ void __launch_bounds__(256) k_hvx_columns(int N, int d, long long P,
                                                      const double2* phi, const double2* dphi,
                                                      const double* r_in, const double* pu_in,
                                                      const double* pr, double2* out) {
  __shared__ double red[2][256];
  const int f = blockIdx.y, k = blockIdx.x, i = threadIdx.x;
  const double2* ph = phi + (size_t)f * N * d;
  const double2* dp = dphi + (size_t)f * N * d;
  const double* fp = pr + (size_t)f * P * kHvPair;
  double gr = 0.0, gi = 0.0, hr = 0.0, hi = 0.0;
  if (i < d) {
    for (int j = 0; j < N; ++j) {
      if (j == k) continue;
      const bool lo = j < k;
      const int a = lo ? j : k, b = lo ? k : j;
      const double* o = fp + (size_t)((long long)a * N - (long long)a * (a + 1) / 2 + (b - a - 1)) * kHvPair;
      const double mr = o[0], mi = lo ? o[1] : -o[1];       // M_jk (conjugate for j > k)
      const double nr = o[2], ni = lo ? o[3] : -o[3];       // dM_jk
      const double2 pj = ph[(size_t)j * d + i], dj = dp[(size_t)j * d + i];
      gr = fma(mr, pj.x, gr); gr = fma(-mi, pj.y, gr);
      gi = fma(mr, pj.y, gi); gi = fma(mi, pj.x, gi);
      hr = fma(nr, pj.x, hr); hr = fma(-ni, pj.y, hr); hr = fma(mr, dj.x, hr); hr = fma(-mi, dj.y, hr);
      hi = fma(nr, pj.y, hi); hi = fma(ni, pj.x, hi); hi = fma(mr, dj.y, hi); hi = fma(mi, dj.x, hi);
    }
    gr *= 2.0; gi *= 2.0; hr *= 2.0; hi *= 2.0;
  }
  const double2 pk = i < d ? ph[(size_t)k * d + i] : make_double2(0.0, 0.0);
  const double2 dk = i < d ? dp[(size_t)k * d + i] : make_double2(0.0, 0.0);
  red[0][i] = i < d ? fma(pk.x, gr, pk.y * gi) : 0.0;
  red[1][i] = i < d ? fma(dk.x, gr, dk.y * gi) + fma(pk.x, hr, pk.y * hi) : 0.0;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (i < st) { red[0][i] += red[0][i + st]; red[1][i] += red[1][i + st]; }
    __syncthreads();
  }
  if (i >= d) return;
  const double rho = red[0][0], drho = red[1][0];
  const long long col = (long long)f * N + k;
  const double inv = 1.0 / r_in[col], pu = pu_in[col];
  const double gradr = (gr - pk.x * rho) * inv, gradi = (gi - pk.y * rho) * inv;
  out[(size_t)col * d + i] = make_double2((hr - dk.x * rho - pk.x * drho) * inv - gradr * pu * inv,
                                          (hi - dk.y * rho - pk.y * drho) * inv - gradi * pu * inv);
}

struct Stack {
  int N, d, L;
  long long n, total;          // 2dN per frame; L frames
  int num_sms;
  cudaStream_t s;
  double *x, *xn, *g, *p, *r, *dv, *bd, *tmp, *gp, *gm;
  double *out, *dots, *coef, *deltas, *hvc;
  int* flag;
  uint32_t* bad;
  void* lse;
  // exact Hessian products: per (frame, column) r and Re(phi^* u), per pair
  // kHvPair doubles, per frame the max x bits, the CTA partials and S, T
  bool exact = false;
  double *hv_r = nullptr, *hv_pu = nullptr, *hv_pairs = nullptr, *hv_part = nullptr,
         *hv_st = nullptr;
  unsigned long long* hv_smax = nullptr;
  // pinned host mirrors
  double *h_coef, *h_out, *h_dots, *h_deltas;
  int* h_flag;
  uint32_t* h_bad;
  int ring = 0;

  unsigned grid() const { return (unsigned)((total + 255) / 256); }

  cudaError_t sync() {
    ring = 0;
    return cudaStreamSynchronize(s);
  }
  // out = a[f] x + b[f] y, frame by frame
  cudaError_t axpby(const std::vector<double>& a, const double* x1, const std::vector<double>& b,
                    const double* y1, double* o) {
    if (ring >= kCoefRing) {
      cudaError_t e = sync();
      if (e != cudaSuccess) return e;
    }
    double* hc = h_coef + (size_t)ring * 2 * L;
    double* dc = coef + (size_t)ring * 2 * L;
    ++ring;
    std::copy(a.begin(), a.end(), hc);
    std::copy(b.begin(), b.end(), hc + L);
    cudaError_t e = cudaMemcpyAsync(dc, hc, 2 * L * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    k_axpby<<<grid(), 256, 0, s>>>(n, total, dc, x1, dc + L, y1, o);
    return cudaGetLastError();
  }
  cudaError_t axpby(double a, const double* x1, const std::vector<double>& b, const double* y1,
                    double* o) {
    return axpby(std::vector<double>(L, a), x1, b, y1, o);
  }
  // per frame x.y, x.z, z.z (z nullable) into q[3f..3f+2]
  cudaError_t dots3(const double* x1, const double* y1, const double* z1, std::vector<double>& q) {
    k_dots<<<L, kDotThreads, 0, s>>>(n, x1, y1, z1, dots);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_dots, dots, 3 * L * sizeof(double),
                                              cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = sync();
    q.assign(h_dots, h_dots + 3 * L);
    return e;
  }
  // the five products of a CG-Steihaug step, q[5f..5f+4] = d.Bd, d.r, p.p, p.d, d.d
  cudaError_t dots5(std::vector<double>& q) {
    k_dots5<<<L, kDotThreads, 0, s>>>(n, dv, bd, r, p, dots);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_dots, dots, 5 * L * sizeof(double),
                                              cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = sync();
    q.assign(h_dots, h_dots + 5 * L);
    return e;
  }
  // the gradient at v with the smoothing parameters already on the device
  // (enqueued only: nothing is read back)
  cudaError_t gradient_async(const double* v, double* grad) {
    return launch_lse_deltas(N, d, L, v, deltas, true, lse, out, grad, num_sms, s);
  }
  // F and s of every frame at v (smoothing parameter per frame), gradient into grad
  cudaError_t objective(const double* v, const std::vector<double>& delta, double* grad,
                        std::vector<double>& F, std::vector<double>* smax) {
    std::copy(delta.begin(), delta.end(), h_deltas);
    cudaError_t e = cudaMemcpyAsync(deltas, h_deltas, L * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = launch_lse_deltas(N, d, L, v, deltas, true, lse, out, grad, num_sms, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h_out, out, 2 * L * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = sync();
    F.resize(L);
    for (int f = 0; f < L; ++f) F[f] = h_out[2 * f];
    if (smax) {
      smax->resize(L);
      for (int f = 0; f < L; ++f) (*smax)[f] = h_out[2 * f + 1];
    }
    return e;
  }
  // o = B u with B the exact Hessian at x (the kernels above; tmp holds phi,
  // gp holds d phi), smoothing parameters of the round already on the device
  cudaError_t hv_exact(const double* u, double* o) {
    const long long P = (long long)N * (N - 1) / 2;
    double2* phi = reinterpret_cast<double2*>(tmp);
    double2* dphi = reinterpret_cast<double2*>(gp);
    k_hvx_cols<<<(unsigned)(((long long)L * N + 127) / 128), 128, 0, s>>>(
        N, d, L, reinterpret_cast<const double2*>(x), reinterpret_cast<const double2*>(u), phi,
        dphi, hv_r, hv_pu);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(hv_smax, 0, L * sizeof(unsigned long long), s)) != cudaSuccess) return e;
    k_hvx_pairs<<<dim3(N - 1, L), 128, 0, s>>>(N, d, P, phi, dphi, hv_pairs, hv_smax);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_hvx_weights<<<dim3(kHvBlocks, L), 256, 0, s>>>(P, deltas, hv_smax, hv_pairs, hv_part);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_hvx_totals<<<(L + 127) / 128, 128, 0, s>>>(L, hv_part, hv_st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_hvx_dm<<<(unsigned)(((long long)L * P + 255) / 256), 256, 0, s>>>(P, L, deltas, hv_st,
                                                                          hv_pairs);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int threads = 32;
    while (threads < d) threads *= 2;   // a power of two for the tree, <= 256 (d <= 256)
    k_hvx_columns<<<dim3(N, L), threads, 0, s>>>(N, d, P, phi, dphi, hv_r, hv_pu, hv_pairs,
                                                 reinterpret_cast<double2*>(o));
    return cudaGetLastError();
  }
  // o = B u, frame by frame: |u| (grad F(x + h u/|u|) - grad F(x - h u/|u|)) / (2h),
  // with the smoothing parameters of the current round already on the device;
  // enqueued only (the coefficients are formed on the device)
  cudaError_t hv(const double* u, double h, double* o) {
    if (exact) return hv_exact(u, o);
    k_dots<<<L, kDotThreads, 0, s>>>(n, u, u, nullptr, dots);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_hv_coef<<<(L + 127) / 128, 128, 0, s>>>(L, dots, h, hvc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_axpby<<<grid(), 256, 0, s>>>(n, total, hvc, x, hvc + L, u, tmp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = gradient_async(tmp, gp)) != cudaSuccess) return e;
    k_axpby<<<grid(), 256, 0, s>>>(n, total, hvc, x, hvc + 2 * L, u, tmp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = gradient_async(tmp, gm)) != cudaSuccess) return e;
    k_axpby<<<grid(), 256, 0, s>>>(n, total, hvc + 3 * L, gp, hvc + 4 * L, gm, o);
    return cudaGetLastError();
  }
  // where want[f]: frame f's columns to unit norm; false if a column was zero
  cudaError_t unit(double* v, const std::vector<int>& want, bool* ok) {
    std::copy(want.begin(), want.end(), h_flag);
    cudaError_t e = cudaMemcpyAsync(flag, h_flag, L * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, L * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    k_unit_columns<<<(unsigned)(((long long)L * N + 127) / 128), 128, 0, s>>>(
        N, d, L, reinterpret_cast<double2*>(v), flag, bad);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = cudaMemcpyAsync(h_bad, bad, L * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = sync();
    *ok = true;
    for (int f = 0; f < L; ++f) if (h_bad[f]) *ok = false;
    return e;
  }
  cudaError_t copy_frames(const std::vector<int>& want, const double* src, double* dst) {
    std::copy(want.begin(), want.end(), h_flag);
    cudaError_t e = cudaMemcpyAsync(flag, h_flag, L * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    k_copy_frames<<<grid(), 256, 0, s>>>(n, total, flag, src, dst);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return sync();   // the flag buffer is rewritten by the next call
  }
};

// tau >= 0 (pos) or <= 0 with |z + tau d| = radius, from z.z, z.d, d.d
__device__ double to_boundary_dev(double zz, double zd, double dd, double radius, bool pos) {
  double disc = zd * zd - dd * (zz - radius * radius);
  if (disc < 0.0) disc = 0.0;
  return pos ? (-zd + sqrt(disc)) / dd : (-zd - sqrt(disc)) / dd;
}
double to_boundary(double zz, double zd, double dd, double radius, bool pos) {
  double disc = zd * zd - dd * (zz - radius * radius);
  if (disc < 0.0) disc = 0.0;
  return pos ? (-zd + std::sqrt(disc)) / dd : (-zd - std::sqrt(disc)) / dd;
}

// CG-Steihaug for the frames with step[f] (the others keep p = 0): the
// paper's Algorithm, frame by frame, on m(p) = g.p + p.Bp / 2, |p| <= radius.
cudaError_t cg_steihaug(Stack& T, double h,
                        const std::vector<double>& radius, const std::vector<double>& eps,
                        const std::vector<int>& step, int maxit, std::vector<double>& m,
                        std::vector<int>& iters, std::vector<int>& status,
                        std::vector<int>& products) {
  const int L = T.L;
  cudaError_t e;
  const size_t bytes = T.total * sizeof(double);
  if ((e = cudaMemsetAsync(T.p, 0, bytes, T.s)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(T.r, T.g, bytes, cudaMemcpyDeviceToDevice, T.s)) != cudaSuccess) return e;
  if ((e = T.axpby(-1.0, T.g, std::vector<double>(L, 0.0), T.g, T.dv)) != cudaSuccess) return e;
  std::vector<double> q;
  if ((e = T.dots3(T.r, T.r, nullptr, q)) != cudaSuccess) return e;
  std::vector<double> rr(L);
  std::vector<int> active(L, 0);
  m.assign(L, 0.0);
  iters.assign(L, 0);
  status.assign(L, 0);
  int n_active = 0;
  for (int f = 0; f < L; ++f) {
    rr[f] = q[3 * f];
    if (step[f] && !(std::sqrt(rr[f]) < eps[f])) { active[f] = 1; ++n_active; }
  }
  for (int it = 0; it < maxit && n_active > 0; ++it) {
    if ((e = T.hv(T.dv, h, T.bd)) != cudaSuccess) return e;
    for (int f = 0; f < L; ++f) products[f] += active[f];
    std::vector<double> dq;
    if ((e = T.dots5(dq)) != cudaSuccess) return e;   // d.Bd, d.r, z.z, z.d, d.d
    std::vector<double> tp(L, 0.0), tr(L, 0.0);
    std::vector<int> cont(L, 0);
    int n_cont = 0;
    for (int f = 0; f < L; ++f) {
      if (!active[f]) continue;
      const double dbd = dq[5 * f], rd = dq[5 * f + 1];
      const double zz = dq[5 * f + 2], zd = dq[5 * f + 3], dd = dq[5 * f + 4];
      if (dbd <= 0.0) {
        const double t1 = to_boundary(zz, zd, dd, radius[f], true);
        const double t2 = to_boundary(zz, zd, dd, radius[f], false);
        const double m1 = m[f] + t1 * rd + 0.5 * t1 * t1 * dbd;
        const double m2 = m[f] + t2 * rd + 0.5 * t2 * t2 * dbd;
        tp[f] = m1 <= m2 ? t1 : t2;
        m[f] = m1 <= m2 ? m1 : m2;
        status[f] = 2; iters[f] = it + 1; active[f] = 0; --n_active;
        continue;
      }
      const double alpha = rr[f] / dbd;
      const double zn2 = zz + 2.0 * alpha * zd + alpha * alpha * dd;
      if (std::sqrt(std::max(zn2, 0.0)) >= radius[f]) {
        const double t = to_boundary(zz, zd, dd, radius[f], true);
        tp[f] = t;
        m[f] += t * rd + 0.5 * t * t * dbd;
        status[f] = 1; iters[f] = it + 1; active[f] = 0; --n_active;
        continue;
      }
      tp[f] = alpha;
      tr[f] = alpha;
      m[f] += alpha * rd + 0.5 * alpha * alpha * dbd;
      cont[f] = 1;
      ++n_cont;
    }
    if ((e = T.axpby(1.0, T.p, tp, T.dv, T.p)) != cudaSuccess) return e;
    if (n_cont == 0) continue;
    if ((e = T.axpby(1.0, T.r, tr, T.bd, T.r)) != cudaSuccess) return e;
    if ((e = T.dots3(T.r, T.r, nullptr, q)) != cudaSuccess) return e;
    std::vector<double> ca(L, 0.0), cb(L, 1.0);
    for (int f = 0; f < L; ++f) {
      if (!cont[f]) continue;
      const double rr_new = q[3 * f];
      if (std::sqrt(rr_new) < eps[f]) {
        status[f] = 0; iters[f] = it + 1; active[f] = 0; --n_active;
        continue;
      }
      ca[f] = -1.0;
      cb[f] = rr_new / rr[f];
      rr[f] = rr_new;
    }
    if ((e = T.axpby(ca, T.r, cb, T.dv, T.dv)) != cudaSuccess) return e;
  }
  for (int f = 0; f < L; ++f)
    if (active[f]) { status[f] = 3; iters[f] = maxit; }
  return cudaSuccess;
}

}  // namespace

// bytes of the exact Hessian products' buffers of the stack (L frames)
size_t hv_exact_bytes(int N, int d, int L) {
  (void)d;
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t P = (size_t)N * (N - 1) / 2;
  return 2 * up((size_t)L * N * sizeof(double)) + up((size_t)L * P * kHvPair * sizeof(double)) +
         up((size_t)L * kHvBlocks * 2 * sizeof(double)) + up((size_t)L * 2 * sizeof(double)) +
         up((size_t)L * sizeof(unsigned long long));
}

size_t tr_device_bytes(int N, int d, int L, int trace_cap, int hessian) {
  const size_t vec = ((size_t)L * 2 * d * N * sizeof(double) + 255) & ~(size_t)255;
  const size_t small = (((size_t)L * (2 + 5 + 2 * kCoefRing + 1 + 5) * sizeof(double) +
                         (size_t)L * (sizeof(int) + sizeof(uint32_t))) + 255) & ~(size_t)255;
  const size_t stack = 10 * vec + small + lse_scratch_bytes(N, d, L, true) +
                       (hessian == 0 ? hv_exact_bytes(N, d, L) : 0);
  // the resident path: per frame mu^2 and three ints, then the trace rows
  const size_t resident = (((size_t)L * 20 + 255) & ~(size_t)255) +
                          (size_t)L * std::max(trace_cap, 0) * sizeof(trstmi_tr_row);
  return std::max(stack, resident);
}

namespace {
int tr_solve_stack(int N, int d, int L, double* v_dev, const trstmi_tr_options& o,
                   void* scratch, int num_sms, cudaStream_t s, TrFrameLog* logs) {
  Stack T;
  T.N = N; T.d = d; T.L = L; T.n = 2LL * d * N; T.total = T.n * L;
  T.num_sms = num_sms; T.s = s;
  const size_t vec = ((size_t)T.total * sizeof(double) + 255) & ~(size_t)255;
  unsigned char* b = static_cast<unsigned char*>(scratch);
  double** vecs[] = {&T.xn, &T.g, &T.p, &T.r, &T.dv, &T.bd, &T.tmp, &T.gp, &T.gm};
  for (int k = 0; k < 9; ++k) *vecs[k] = reinterpret_cast<double*>(b + k * vec);
  double* small = reinterpret_cast<double*>(b + 9 * vec);
  T.out = small;
  T.dots = T.out + 2 * L;
  T.coef = T.dots + 5 * L;
  T.deltas = T.coef + 2 * (size_t)kCoefRing * L;
  T.hvc = T.deltas + L;
  T.flag = reinterpret_cast<int*>(T.hvc + 5 * L);
  T.bad = reinterpret_cast<uint32_t*>(T.flag + L);
  const size_t small_bytes = (((size_t)L * (2 + 5 + 2 * kCoefRing + 1 + 5) * sizeof(double) +
                               (size_t)L * (sizeof(int) + sizeof(uint32_t))) + 255) & ~(size_t)255;
  T.lse = b + 9 * vec + small_bytes;
  T.x = v_dev;
  T.exact = o.hessian == 0;
  if (T.exact) {
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t P = (size_t)N * (N - 1) / 2;
    unsigned char* h = static_cast<unsigned char*>(T.lse) + lse_scratch_bytes(N, d, L, true);
    T.hv_r = reinterpret_cast<double*>(h); h += up((size_t)L * N * sizeof(double));
    T.hv_pu = reinterpret_cast<double*>(h); h += up((size_t)L * N * sizeof(double));
    T.hv_pairs = reinterpret_cast<double*>(h); h += up((size_t)L * P * kHvPair * sizeof(double));
    T.hv_part = reinterpret_cast<double*>(h); h += up((size_t)L * kHvBlocks * 2 * sizeof(double));
    T.hv_st = reinterpret_cast<double*>(h); h += up((size_t)L * 2 * sizeof(double));
    T.hv_smax = reinterpret_cast<unsigned long long*>(h);
  }
  void* pinned = nullptr;
  const size_t pinned_bytes = (size_t)L * (2 * kCoefRing + 2 + 5 + 1) * sizeof(double) +
                              (size_t)L * (sizeof(int) + sizeof(uint32_t));
  if (cudaMallocHost(&pinned, pinned_bytes) != cudaSuccess) return TRSTMI_ENOMEM;
  T.h_coef = static_cast<double*>(pinned);
  T.h_out = T.h_coef + 2 * (size_t)kCoefRing * L;
  T.h_dots = T.h_out + 2 * L;
  T.h_deltas = T.h_dots + 5 * L;
  T.h_flag = reinterpret_cast<int*>(T.h_deltas + L);
  T.h_bad = reinterpret_cast<uint32_t*>(T.h_flag + L);

  std::vector<int> stage(L, 0), it(L, 0), finished(L, 0), all(L, 1);
  std::vector<double> radius(L, o.radius0);
  std::vector<int> products(L, 0);
  auto advance = [&](int f) {
    ++stage[f]; it[f] = 0; radius[f] = o.radius0;
    if (stage[f] >= o.n_delta) finished[f] = 1;
  };
  int rc = TRSTMI_OK;
  bool ok = true;
  cudaError_t e = T.unit(T.x, all, &ok);
  if (e == cudaSuccess && !ok) rc = TRSTMI_EINVAL;
  if (o.max_outer == 0)
    for (int f = 0; f < L; ++f) finished[f] = 1;
  while (e == cudaSuccess && rc == TRSTMI_OK) {
    int n_open = 0;
    for (int f = 0; f < L; ++f) n_open += !finished[f];
    if (n_open == 0) break;
    std::vector<double> delta(L), F, smax, Fn, gq, pq;
    for (int f = 0; f < L; ++f) delta[f] = o.delta[std::min(stage[f], o.n_delta - 1)];
    if ((e = T.objective(T.x, delta, T.g, F, &smax)) != cudaSuccess) break;
    if ((e = T.dots3(T.g, T.g, nullptr, gq)) != cudaSuccess) break;
    std::vector<int> step(L, 0);
    std::vector<double> gn(L), eps(L, 0.0);
    int n_step = 0;
    for (int f = 0; f < L; ++f) {
      if (finished[f]) continue;
      gn[f] = std::sqrt(gq[3 * f]);
      if (gn[f] <= o.gtol) { advance(f); continue; }
      step[f] = 1;
      ++n_step;
      eps[f] = std::min(0.5, std::sqrt(gn[f])) * gn[f];
    }
    if (n_step == 0) continue;
    std::vector<double> m;
    std::vector<int> cgit, cgst;
    // the round's smoothing parameters stay on the device for the Hessian products
    if ((e = cg_steihaug(T, o.fd_step, radius, eps, step, o.max_cg, m, cgit, cgst,
                         products)) != cudaSuccess)
      break;
    if ((e = T.dots3(T.p, T.p, nullptr, pq)) != cudaSuccess) break;
    if ((e = T.axpby(1.0, T.x, std::vector<double>(L, 1.0), T.p, T.xn)) != cudaSuccess) break;
    if ((e = T.objective(T.xn, delta, nullptr, Fn, nullptr)) != cudaSuccess) break;
    std::vector<int> acc(L, 0);
    int n_acc = 0;
    for (int f = 0; f < L; ++f) {
      if (!step[f]) continue;
      const double pn = std::sqrt(pq[3 * f]);
      const double pred = -m[f];
      const double rho = pred > 0.0 ? (F[f] - Fn[f]) / pred : -1.0;
      const double r_used = radius[f];
      if (rho < 0.25) radius[f] *= 0.25;
      else if (rho > 0.75 && pn >= (1.0 - 1e-12) * radius[f])
        radius[f] = std::min(2.0 * radius[f], o.radius_max);
      acc[f] = rho > o.eta ? 1 : 0;
      n_acc += acc[f];
      if (logs && logs[f].rows && logs[f].n < logs[f].cap) {
        trstmi_tr_row& r = logs[f].rows[logs[f].n];
        r.stage = stage[f]; r.iter = it[f]; r.F = F[f]; r.s = smax[f]; r.gnorm = gn[f];
        r.radius = r_used; r.rho = rho; r.step_norm = pn; r.pred = pred;
        r.cg_iters = cgit[f]; r.cg_status = cgst[f]; r.accepted = acc[f]; r.reserved = 0;
      }
      if (logs) ++logs[f].n;
      ++it[f];
      if (it[f] >= o.max_outer || radius[f] < 1e-14) advance(f);
    }
    if (n_acc > 0) {
      if ((e = T.copy_frames(acc, T.xn, T.x)) != cudaSuccess) break;
      if ((e = T.unit(T.x, acc, &ok)) != cudaSuccess) break;
      if (!ok) rc = TRSTMI_EINVAL;
    }
  }
  // the coherence each frame ended with (its largest |G_jk|^2, binary64)
  if (e == cudaSuccess && rc == TRSTMI_OK && logs) {
    std::vector<double> delta(L, o.delta[o.n_delta - 1]), F, smax;
    e = T.objective(T.x, delta, nullptr, F, &smax);
    if (e == cudaSuccess)
      for (int f = 0; f < L; ++f) logs[f].mu2 = smax[f];
  }
  if (logs)
    for (int f = 0; f < L; ++f) logs[f].hv_products = products[f];
  cudaFreeHost(pinned);
  if (rc != TRSTMI_OK) return rc;
  return e == cudaSuccess ? TRSTMI_OK : TRSTMI_ECUDA;
}

// ------------------------------------------------- frames resident in one CTA
// For frames small enough to live in shared memory (the paper's Table 2 shapes
// up to d = 9, N = 81), one CTA runs a frame's whole procedure: every vector in
// shared memory, F and its gradient formed by the CTA (pairs j < k spread over
// the threads, a fixed order in every sum), inner products by a fixed tree, the
// algorithms' scalar logic computed by every thread from the same reduced
// values.  No host round trip and no other frame to wait for: L trials are L
// independent CTAs.  Every loop is bounded by the options (stages x max_outer x
// max_cg).

constexpr int kResThreads = 256;

struct ResArgs {
  int N, d, P;                     // P = N(N-1)/2 pairs
  double* v;                       // L frames, N x d complex (in / out)
  trstmi_tr_options o;
  trstmi_tr_row* rows;             // L x cap, or null
  int cap;
  int* n_rows;                     // L
  double* mu2;                     // L: max |G_jk|^2 at the end
  int* hv;                         // L: Hessian products
  int* bad;                        // L: a zero column was met
  int exact;                       // 1: exact Hessian products, 0: central differences
};

// Shared memory of one frame: the vectors (2dN doubles each), per column 1/r
// and rho = Re(phi_k^* g_k), per pair G, the softmax weight w and (exact
// products) dG, later dM; a reduction buffer of half the CTA; the first
// column index of every pair.  Central differences need two gradients
// (gp, gm) instead of the pair arrays dM.
constexpr int kResRed = kResThreads / 2;
struct ResSmem {
  double *x, *xn, *g, *p, *r, *dv, *bd, *gp, *gm, *phi, *rn, *rho, *Gre, *Gim, *W, *dMre, *dMim,
      *red;
  unsigned short* pj;
};

size_t res_doubles(int N, int d, bool exact) {
  const size_t n = 2 * (size_t)d * N, P = (size_t)N * (N - 1) / 2;
  return 8 * n + 2 * (size_t)N + 3 * P + kResRed + (exact ? 2 * P : 2 * n);
}
size_t res_smem_bytes(int N, int d, bool exact) {
  const size_t P = (size_t)N * (N - 1) / 2;
  return res_doubles(N, d, exact) * sizeof(double) + ((P * sizeof(unsigned short) + 15) & ~15ull);
}

// pair q = (j, k), j < k, numbered row by row: k from q and j
__device__ __forceinline__ int res_pair_k(int q, int j, int N) {
  return q - (j * N - j * (j + 1) / 2) + j + 1;
}

// sum over the CTA of each thread's v, the same order every call (thread t
// and t + kResRed first, then a tree); all threads get the result
__device__ double res_sum(double v, double* red) {
  __syncthreads();
  if (threadIdx.x < kResRed) red[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x >= kResRed) red[threadIdx.x - kResRed] += v;
  __syncthreads();
  for (int st = kResRed / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  const double out = red[0];
  __syncthreads();
  return out;
}
__device__ double res_max(double v, double* red) {
  __syncthreads();
  if (threadIdx.x < kResRed) red[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x >= kResRed) red[threadIdx.x - kResRed] = fmax(red[threadIdx.x - kResRed], v);
  __syncthreads();
  for (int st = kResRed / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + st]);
    __syncthreads();
  }
  const double out = red[0];
  __syncthreads();
  return out;
}
__device__ double res_dot(const double* a, const double* b, int n, double* red) {
  double t = 0.0;
  for (int i = threadIdx.x; i < n; i += kResThreads) t += a[i] * b[i];
  return res_sum(t, red);
}
// o = a x + b y over n entries
__device__ void res_axpby(double a, const double* x, double b, const double* y, double* o, int n) {
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += kResThreads) o[i] = a * x[i] + b * y[i];
  __syncthreads();
}

// F_{s,delta} and s at v; the gradient into gout when it is not null.
// Returns false (in every thread) if a column of v is zero.
//
// Binary64 runs at about two fused multiply-adds per clock per SM on this
// part, so the pass is written for the fewest binary64 operations: one
// reciprocal per column and one of delta and of the sum (no division per
// entry or pair), one exponential per pair (kept in W), and the weighted
// Gram M = w (.) G formed once per pair, so that the gradient's inner loop is
// four fused multiply-adds per (k, i, j).  The complex products are written
// as explicit fma chains: "acc += a*b + c*d" would compile to a multiply, a
// fused multiply-add and an add, three binary64 instructions for two.
__device__ bool res_eval(const ResArgs& a, ResSmem& S, const double* v, double delta,
                         double* gout, double* F, double* smax) {
  const int N = a.N, d = a.d, P = a.P;
  __syncthreads();
  double zero = 0.0;
  for (int k = threadIdx.x; k < N; k += kResThreads) {
    double q = 0.0;
    for (int i = 0; i < d; ++i) {
      const double re = v[2 * (k * d + i)], im = v[2 * (k * d + i) + 1];
      q = fma(re, re, q);
      q = fma(im, im, q);
    }
    if (!(q > 0.0)) zero = 1.0;
    const double r = sqrt(q), inv = 1.0 / r;
    S.rn[k] = inv;
    for (int i = 0; i < d; ++i) {
      S.phi[2 * (k * d + i)] = v[2 * (k * d + i)] * inv;
      S.phi[2 * (k * d + i) + 1] = v[2 * (k * d + i) + 1] * inv;
    }
  }
  if (res_max(zero, S.red) > 0.0) return false;
  // G_jk = sum_i conj(phi_ij) phi_ik and x = |G_jk|^2 for every pair
  double hi = 0.0;
  for (int q = threadIdx.x; q < P; q += kResThreads) {
    const int j = S.pj[q], k = res_pair_k(q, j, N);
    double gr = 0.0, gi = 0.0;
    for (int i = 0; i < d; ++i) {
      const double ar = S.phi[2 * (j * d + i)], ai = S.phi[2 * (j * d + i) + 1];
      const double br = S.phi[2 * (k * d + i)], bi = S.phi[2 * (k * d + i) + 1];
      gr = fma(ar, br, gr);
      gr = fma(ai, bi, gr);
      gi = fma(ar, bi, gi);
      gi = fma(-ai, br, gi);
    }
    S.Gre[q] = gr;
    S.Gim[q] = gi;
    const double x = gr * gr + gi * gi;
    S.W[q] = x;
    hi = fmax(hi, x);
  }
  const double s = res_max(hi, S.red);
  const double inv_delta = 1.0 / delta;
  double e = 0.0;
  for (int q = threadIdx.x; q < P; q += kResThreads) {
    const double t = exp((S.W[q] - s) * inv_delta);
    S.W[q] = t;
    e += t;
  }
  const double Ssum = res_sum(e, S.red);
  *F = s + delta * log(Ssum);
  *smax = s;
  if (!gout) return true;
  // the softmax weights w = exp((x - s)/delta) / Ssum (G is kept: the exact
  // Hessian products need it); M = w (.) G is formed where it is used
  const double inv_sum = 1.0 / Ssum;
  for (int q = threadIdx.x; q < P; q += kResThreads) S.W[q] *= inv_sum;
  __syncthreads();
  // g_k = 2 sum_{j != k} M_jk phi_j (M Hermitian: M_jk = conj(M_kj) for j > k),
  // j ascending, then the projection
  const int half = d * N;
  for (int t = threadIdx.x; t < half; t += kResThreads) {
    const int k = t / d, i = t - k * d;
    double gr = 0.0, gi = 0.0;
    for (int j = 0; j < k; ++j) {
      const int q = j * N - j * (j + 1) / 2 + (k - j - 1);
      const double mr = S.W[q] * S.Gre[q], mi = S.W[q] * S.Gim[q];
      const double pr = S.phi[2 * (j * d + i)], pi = S.phi[2 * (j * d + i) + 1];
      gr = fma(mr, pr, gr);
      gr = fma(-mi, pi, gr);
      gi = fma(mr, pi, gi);
      gi = fma(mi, pr, gi);
    }
    const int base = k * N - k * (k + 1) / 2 - k - 1;
    for (int j = k + 1; j < N; ++j) {
      const int q = base + j;
      const double mr = S.W[q] * S.Gre[q], mi = S.W[q] * S.Gim[q];
      const double pr = S.phi[2 * (j * d + i)], pi = S.phi[2 * (j * d + i) + 1];
      gr = fma(mr, pr, gr);
      gr = fma(mi, pi, gr);
      gi = fma(mr, pi, gi);
      gi = fma(-mi, pr, gi);
    }
    gout[2 * (k * d + i)] = 2.0 * gr;
    gout[2 * (k * d + i) + 1] = 2.0 * gi;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < N; k += kResThreads) {
    double rad = 0.0;
    for (int i = 0; i < d; ++i) {
      rad = fma(S.phi[2 * (k * d + i)], gout[2 * (k * d + i)], rad);
      rad = fma(S.phi[2 * (k * d + i) + 1], gout[2 * (k * d + i) + 1], rad);
    }
    const double inv = S.rn[k];
    S.rho[k] = rad;
    for (int i = 0; i < d; ++i) {
      gout[2 * (k * d + i)] = (gout[2 * (k * d + i)] - S.phi[2 * (k * d + i)] * rad) * inv;
      gout[2 * (k * d + i) + 1] =
          (gout[2 * (k * d + i) + 1] - S.phi[2 * (k * d + i) + 1] * rad) * inv;
    }
  }
  __syncthreads();
  return true;
}

// out = B u, B the exact Hessian of F_{s,delta} at S.x, from the state the
// last res_eval(S.x, gradient into S.g) left: phi, 1/r, rho, G and w.  The
// chain rule of the stack's kernels above (k_hvx_*), with d phi in S.xn and
// dG, then dM, in the pair arrays.
__device__ void res_hv_exact(const ResArgs& a, ResSmem& S, const double* u, double* out,
                             double delta) {
  const int N = a.N, d = a.d, P = a.P;
  __syncthreads();
  double* dphi = S.xn;
  for (int k = threadIdx.x; k < N; k += kResThreads) {
    double pu = 0.0;
    for (int i = 0; i < d; ++i) {
      pu = fma(S.phi[2 * (k * d + i)], u[2 * (k * d + i)], pu);
      pu = fma(S.phi[2 * (k * d + i) + 1], u[2 * (k * d + i) + 1], pu);
    }
    const double inv = S.rn[k];
    for (int c = 0; c < 2 * d; ++c)
      dphi[2 * k * d + c] = (u[2 * k * d + c] - S.phi[2 * k * d + c] * pu) * inv;
  }
  __syncthreads();
  // dG and T = sum w dx, dx = 2 Re(conj(G) dG)
  double tpart = 0.0;
  for (int q = threadIdx.x; q < P; q += kResThreads) {
    const int j = S.pj[q], k = res_pair_k(q, j, N);
    double hr = 0.0, hi = 0.0;
    for (int i = 0; i < d; ++i) {
      const double ar = S.phi[2 * (j * d + i)], ai = S.phi[2 * (j * d + i) + 1];
      const double br = S.phi[2 * (k * d + i)], bi = S.phi[2 * (k * d + i) + 1];
      const double dar = dphi[2 * (j * d + i)], dai = dphi[2 * (j * d + i) + 1];
      const double dbr = dphi[2 * (k * d + i)], dbi = dphi[2 * (k * d + i) + 1];
      hr = fma(dar, br, hr); hr = fma(dai, bi, hr); hr = fma(ar, dbr, hr); hr = fma(ai, dbi, hr);
      hi = fma(dar, bi, hi); hi = fma(-dai, br, hi); hi = fma(ar, dbi, hi); hi = fma(-ai, dbr, hi);
    }
    S.dMre[q] = hr;
    S.dMim[q] = hi;
    tpart = fma(S.W[q], 2.0 * (S.Gre[q] * hr + S.Gim[q] * hi), tpart);
  }
  const double T = res_sum(tpart, S.red);
  const double inv_delta = 1.0 / delta;
  for (int q = threadIdx.x; q < P; q += kResThreads) {
    const double gr = S.Gre[q], gi = S.Gim[q], hr = S.dMre[q], hi = S.dMim[q], w = S.W[q];
    const double dw = w * (2.0 * (gr * hr + gi * hi) - T) * inv_delta;
    S.dMre[q] = fma(dw, gr, w * hr);
    S.dMim[q] = fma(dw, gi, w * hi);
  }
  __syncthreads();
  // dg_k = 2 sum_{j != k} (dM_jk phi_j + M_jk d phi_j), j ascending
  const int half = d * N;
  for (int t = threadIdx.x; t < half; t += kResThreads) {
    const int k = t / d, i = t - k * d;
    double hr = 0.0, hi = 0.0;
    for (int j = 0; j < N; ++j) {
      if (j == k) continue;
      const bool lo = j < k;
      const int q = lo ? j * N - j * (j + 1) / 2 + (k - j - 1) : k * N - k * (k + 1) / 2 + (j - k - 1);
      const double w = S.W[q];
      const double mr = w * S.Gre[q], mi = lo ? w * S.Gim[q] : -(w * S.Gim[q]);
      const double nr = S.dMre[q], ni = lo ? S.dMim[q] : -S.dMim[q];
      const double pr = S.phi[2 * (j * d + i)], pi = S.phi[2 * (j * d + i) + 1];
      const double qr = dphi[2 * (j * d + i)], qi = dphi[2 * (j * d + i) + 1];
      hr = fma(nr, pr, hr); hr = fma(-ni, pi, hr); hr = fma(mr, qr, hr); hr = fma(-mi, qi, hr);
      hi = fma(nr, pi, hi); hi = fma(ni, pr, hi); hi = fma(mr, qi, hi); hi = fma(mi, qr, hi);
    }
    out[2 * (k * d + i)] = 2.0 * hr;
    out[2 * (k * d + i) + 1] = 2.0 * hi;
  }
  __syncthreads();
  // the projection through the normalisation: g_k = r_k grad_k + phi_k rho_k,
  // d rho = Re(d phi^* g + phi^* dg), (B u)_k = (dg - d phi rho - phi d rho)/r
  // - grad d r / r with d r = Re(phi^* u)
  for (int k = threadIdx.x; k < N; k += kResThreads) {
    double q2 = 0.0, pu = 0.0;
    for (int i = 0; i < d; ++i) {
      const double re = S.x[2 * (k * d + i)], im = S.x[2 * (k * d + i) + 1];
      q2 = fma(re, re, q2);
      q2 = fma(im, im, q2);
      pu = fma(S.phi[2 * (k * d + i)], u[2 * (k * d + i)], pu);
      pu = fma(S.phi[2 * (k * d + i) + 1], u[2 * (k * d + i) + 1], pu);
    }
    const double r = sqrt(q2), inv = S.rn[k], rho = S.rho[k];
    double drho = 0.0;
    for (int c = 0; c < 2 * d; ++c) {
      const double graw = fma(r, S.g[2 * k * d + c], S.phi[2 * k * d + c] * rho);
      drho = fma(dphi[2 * k * d + c], graw, drho);
      drho = fma(S.phi[2 * k * d + c], out[2 * k * d + c], drho);
    }
    for (int c = 0; c < 2 * d; ++c) {
      const double dg = out[2 * k * d + c];
      out[2 * k * d + c] =
          (dg - dphi[2 * k * d + c] * rho - S.phi[2 * k * d + c] * drho) * inv -
          S.g[2 * k * d + c] * pu * inv;
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kResThreads, 1) k_tr_resident(const ResArgs a) {
  extern __shared__ __align__(16) double sm[];
  const int f = blockIdx.x;
  const int N = a.N, d = a.d, P = a.P, n = 2 * d * N;
  const trstmi_tr_options& o = a.o;
  ResSmem S;
  double* c = sm;
  S.x = c; c += n; S.xn = c; c += n; S.g = c; c += n; S.p = c; c += n; S.r = c; c += n;
  S.dv = c; c += n; S.bd = c; c += n; S.phi = c; c += n;
  S.rn = c; c += N; S.rho = c; c += N; S.Gre = c; c += P; S.Gim = c; c += P; S.W = c; c += P;
  S.red = c; c += kResRed;
  S.gp = S.gm = S.dMre = S.dMim = nullptr;
  if (a.exact) {
    S.dMre = c; c += P; S.dMim = c; c += P;
  } else {
    S.gp = c; c += n; S.gm = c; c += n;
  }
  S.pj = reinterpret_cast<unsigned short*>(c);
  for (int q = threadIdx.x; q < P; q += kResThreads) {
    int j = 0, rem = q;
    while (rem >= N - 1 - j) { rem -= N - 1 - j; ++j; }
    S.pj[q] = (unsigned short)j;
  }
  double* vf = a.v + (size_t)f * n;
  for (int i = threadIdx.x; i < n; i += kResThreads) S.x[i] = vf[i];
  __syncthreads();
  // columns to unit norm
  bool ok = true;
  {
    double F0, s0;
    ok = res_eval(a, S, S.x, 1.0, nullptr, &F0, &s0);
    if (ok) {
      for (int i = threadIdx.x; i < n; i += kResThreads) S.x[i] = S.phi[i];
      __syncthreads();
    }
  }
  int rows = 0, products = 0;
  trstmi_tr_row* trace = a.rows ? a.rows + (size_t)f * a.cap : nullptr;
  const double h = o.fd_step;
  for (int k = 0; k < o.n_delta && ok; ++k) {
    const double delta = o.delta[k];
    double radius = o.radius0;
    for (int it = 0; it < o.max_outer && ok; ++it) {
      double F, smax, Fn, sn;
      ok = res_eval(a, S, S.x, delta, S.g, &F, &smax);
      if (!ok) break;
      const double gn = sqrt(res_dot(S.g, S.g, n, S.red));
      if (gn <= o.gtol) break;
      const double eps = fmin(0.5, sqrt(gn)) * gn;
      // CG-Steihaug (the paper's Algorithm, Nocedal and Wright Alg. 7.2)
      res_axpby(0.0, S.g, 0.0, S.g, S.p, n);
      res_axpby(1.0, S.g, 0.0, S.g, S.r, n);
      res_axpby(-1.0, S.g, 0.0, S.g, S.dv, n);
      double m = 0.0, rr = res_dot(S.r, S.r, n, S.red);
      int st = 3, cgit = 0;
      if (sqrt(rr) < eps) {
        st = 0;
      } else {
        for (cgit = 0; cgit < o.max_cg; ++cgit) {
          if (a.exact) {
            // B d with the exact Hessian at the iterate
            res_hv_exact(a, S, S.dv, S.bd, delta);
          } else {
            // B d by a central difference of the gradient
            const double nu = sqrt(res_dot(S.dv, S.dv, n, S.red));
            const double step = nu > 0.0 ? h / nu : 0.0, cq = nu > 0.0 ? nu / (2.0 * h) : 0.0;
            double Ft, st2;
            res_axpby(1.0, S.x, step, S.dv, S.xn, n);
            ok = res_eval(a, S, S.xn, delta, S.gp, &Ft, &st2);
            res_axpby(1.0, S.x, -step, S.dv, S.xn, n);
            ok = ok && res_eval(a, S, S.xn, delta, S.gm, &Ft, &st2);
            if (!ok) break;
            res_axpby(cq, S.gp, -cq, S.gm, S.bd, n);
          }
          ++products;
          const double dbd = res_dot(S.dv, S.bd, n, S.red), rd = res_dot(S.dv, S.r, n, S.red);
          const double zz = res_dot(S.p, S.p, n, S.red), zd = res_dot(S.p, S.dv, n, S.red);
          const double dd = res_dot(S.dv, S.dv, n, S.red);
          if (dbd <= 0.0) {
            const double t1 = to_boundary_dev(zz, zd, dd, radius, true);
            const double t2 = to_boundary_dev(zz, zd, dd, radius, false);
            const double m1 = m + t1 * rd + 0.5 * t1 * t1 * dbd;
            const double m2 = m + t2 * rd + 0.5 * t2 * t2 * dbd;
            res_axpby(1.0, S.p, m1 <= m2 ? t1 : t2, S.dv, S.p, n);
            m = m1 <= m2 ? m1 : m2;
            st = 2; ++cgit;
            break;
          }
          const double alpha = rr / dbd;
          const double zn2 = zz + 2.0 * alpha * zd + alpha * alpha * dd;
          if (sqrt(fmax(zn2, 0.0)) >= radius) {
            const double t = to_boundary_dev(zz, zd, dd, radius, true);
            res_axpby(1.0, S.p, t, S.dv, S.p, n);
            m += t * rd + 0.5 * t * t * dbd;
            st = 1; ++cgit;
            break;
          }
          res_axpby(1.0, S.p, alpha, S.dv, S.p, n);
          res_axpby(1.0, S.r, alpha, S.bd, S.r, n);
          m += alpha * rd + 0.5 * alpha * alpha * dbd;
          const double rr_new = res_dot(S.r, S.r, n, S.red);
          if (sqrt(rr_new) < eps) { st = 0; ++cgit; break; }
          res_axpby(-1.0, S.r, rr_new / rr, S.dv, S.dv, n);
          rr = rr_new;
        }
      }
      if (!ok) break;
      const double pn = sqrt(res_dot(S.p, S.p, n, S.red));
      res_axpby(1.0, S.x, 1.0, S.p, S.xn, n);
      ok = res_eval(a, S, S.xn, delta, nullptr, &Fn, &sn);
      if (!ok) break;
      const double pred = -m;
      const double rho = pred > 0.0 ? (F - Fn) / pred : -1.0;
      const double r_used = radius;
      if (rho < 0.25) radius *= 0.25;
      else if (rho > 0.75 && pn >= (1.0 - 1e-12) * radius) radius = fmin(2.0 * radius, o.radius_max);
      const bool acc = rho > o.eta;
      if (acc) {
        // V <- V + p with unit columns: the phi of the last evaluation
        for (int i = threadIdx.x; i < n; i += kResThreads) S.x[i] = S.phi[i];
        __syncthreads();
      }
      if (trace && rows < a.cap && threadIdx.x == 0) {
        trstmi_tr_row& w = trace[rows];
        w.stage = k; w.iter = it; w.F = F; w.s = smax; w.gnorm = gn; w.radius = r_used;
        w.rho = rho; w.step_norm = pn; w.pred = pred; w.cg_iters = cgit; w.cg_status = st;
        w.accepted = acc ? 1 : 0; w.reserved = 0;
      }
      ++rows;
      if (radius < 1e-14) break;
    }
  }
  double Fe = 0.0, se = 0.0;
  if (ok) ok = res_eval(a, S, S.x, o.delta[o.n_delta - 1], nullptr, &Fe, &se);
  for (int i = threadIdx.x; i < n; i += kResThreads) vf[i] = S.x[i];
  if (threadIdx.x == 0) {
    a.n_rows[f] = rows;
    a.mu2[f] = se;
    a.hv[f] = products;
    a.bad[f] = ok ? 0 : 1;
  }
}

}  // namespace

bool tr_resident_fits(int N, int d, bool exact) {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return false;
  // the kernel has no static shared memory: the whole opt-in size is dynamic
  return N <= 65535 && res_smem_bytes(N, d, exact) <= (size_t)optin;
}

int tr_solve_device(int N, int d, int L, double* v_dev, const trstmi_tr_options& o,
                    void* scratch, int num_sms, cudaStream_t s, TrFrameLog* logs) {
  const bool exact = o.hessian == 0;
  const bool resident = o.path == 2 || (o.path == 0 && tr_resident_fits(N, d, exact));
  if (!resident) return tr_solve_stack(N, d, L, v_dev, o, scratch, num_sms, s, logs);
  if (!tr_resident_fits(N, d, exact)) return TRSTMI_EUNSUPPORTED;
  int cap = 0;
  for (int f = 0; f < L && logs; ++f) cap = std::max(cap, logs[f].rows ? logs[f].cap : 0);
  // results in the scratch array: L ints x 3 and L doubles, then the rows
  unsigned char* b = static_cast<unsigned char*>(scratch);
  ResArgs a;
  a.N = N; a.d = d; a.P = N * (N - 1) / 2; a.v = v_dev; a.o = o; a.cap = cap;
  a.exact = exact ? 1 : 0;
  a.mu2 = reinterpret_cast<double*>(b);
  a.n_rows = reinterpret_cast<int*>(a.mu2 + L);
  a.hv = a.n_rows + L;
  a.bad = a.hv + L;
  a.rows = cap > 0 ? reinterpret_cast<trstmi_tr_row*>(b + (((size_t)L * 20 + 255) & ~(size_t)255))
                   : nullptr;
  const size_t smem = res_smem_bytes(N, d, exact);
  cudaError_t e = cudaFuncSetAttribute(k_tr_resident, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e == cudaSuccess) {
    k_tr_resident<<<L, kResThreads, smem, s>>>(a);
    e = cudaGetLastError();
  }
  std::vector<double> mu2(L);
  std::vector<int> ints(3 * (size_t)L);
  if (e == cudaSuccess) e = cudaMemcpyAsync(mu2.data(), a.mu2, L * sizeof(double),
                                            cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ints.data(), a.n_rows, 3 * L * sizeof(int),
                                            cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return TRSTMI_ECUDA;
  for (int f = 0; f < L; ++f)
    if (ints[2 * L + f]) return TRSTMI_EINVAL;
  if (logs) {
    for (int f = 0; f < L; ++f) {
      logs[f].n = ints[f];
      logs[f].mu2 = mu2[f];
      logs[f].hv_products = ints[L + f];
      if (logs[f].rows && cap > 0) {
        const int k = std::min(ints[f], std::min(cap, logs[f].cap));
        if (k > 0 && cudaMemcpy(logs[f].rows, a.rows + (size_t)f * cap, k * sizeof(trstmi_tr_row),
                                cudaMemcpyDeviceToHost) != cudaSuccess)
          return TRSTMI_ECUDA;
      }
    }
  }
  return TRSTMI_OK;
}

}  // namespace trstmi
