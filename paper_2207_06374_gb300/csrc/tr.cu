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
// it follows alone (L = 1).  Hessian products are central differences of the
// exact gradient (Hessian-free, as in Nocedal and Wright's Newton-CG), all in
// binary64.
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

struct Stack {
  int N, d, L;
  long long n, total;          // 2dN per frame; L frames
  int num_sms;
  cudaStream_t s;
  double *x, *xn, *g, *p, *r, *dv, *bd, *tmp, *gp, *gm;
  double *out, *dots, *coef, *deltas;
  int* flag;
  uint32_t* bad;
  void* lse;
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
  cudaError_t norms(const double* x1, std::vector<double>& nrm) {
    std::vector<double> q;
    cudaError_t e = dots3(x1, x1, nullptr, q);
    nrm.resize(L);
    for (int f = 0; f < L; ++f) nrm[f] = std::sqrt(q[3 * f]);
    return e;
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
  // o = B u, frame by frame: |u| (grad F(x + h u/|u|) - grad F(x - h u/|u|)) / (2h)
  cudaError_t hv(const double* u, const std::vector<double>& delta, double h, double* o) {
    std::vector<double> nu, step(L), c(L), F;
    cudaError_t e = norms(u, nu);
    if (e != cudaSuccess) return e;
    for (int f = 0; f < L; ++f) {
      step[f] = nu[f] > 0.0 ? h / nu[f] : 0.0;
      c[f] = nu[f] > 0.0 ? nu[f] / (2.0 * h) : 0.0;
    }
    std::vector<double> nstep(L), nc(L);
    for (int f = 0; f < L; ++f) { nstep[f] = -step[f]; nc[f] = -c[f]; }
    if ((e = axpby(1.0, x, step, u, tmp)) != cudaSuccess) return e;
    if ((e = objective(tmp, delta, gp, F, nullptr)) != cudaSuccess) return e;
    if ((e = axpby(1.0, x, nstep, u, tmp)) != cudaSuccess) return e;
    if ((e = objective(tmp, delta, gm, F, nullptr)) != cudaSuccess) return e;
    return axpby(c, gp, nc, gm, o);
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
double to_boundary(double zz, double zd, double dd, double radius, bool pos) {
  double disc = zd * zd - dd * (zz - radius * radius);
  if (disc < 0.0) disc = 0.0;
  return pos ? (-zd + std::sqrt(disc)) / dd : (-zd - std::sqrt(disc)) / dd;
}

// CG-Steihaug for the frames with step[f] (the others keep p = 0): the
// paper's Algorithm, frame by frame, on m(p) = g.p + p.Bp / 2, |p| <= radius.
cudaError_t cg_steihaug(Stack& T, const std::vector<double>& delta, double h,
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
    if ((e = T.hv(T.dv, delta, h, T.bd)) != cudaSuccess) return e;
    for (int f = 0; f < L; ++f) products[f] += active[f];
    std::vector<double> dq, zq;
    if ((e = T.dots3(T.dv, T.bd, T.r, dq)) != cudaSuccess) return e;   // d.Bd, d.r
    if ((e = T.dots3(T.p, T.p, T.dv, zq)) != cudaSuccess) return e;    // z.z, z.d, d.d
    std::vector<double> tp(L, 0.0), tr(L, 0.0);
    std::vector<int> cont(L, 0);
    int n_cont = 0;
    for (int f = 0; f < L; ++f) {
      if (!active[f]) continue;
      const double dbd = dq[3 * f], rd = dq[3 * f + 1];
      const double zz = zq[3 * f], zd = zq[3 * f + 1], dd = zq[3 * f + 2];
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

size_t tr_device_bytes(int N, int d, int L) {
  const size_t vec = ((size_t)L * 2 * d * N * sizeof(double) + 255) & ~(size_t)255;
  const size_t small = (((size_t)L * (2 + 3 + 2 * kCoefRing + 1) * sizeof(double) +
                         (size_t)L * (sizeof(int) + sizeof(uint32_t))) + 255) & ~(size_t)255;
  return 10 * vec + small + lse_scratch_bytes(N, d, L, true);
}

int tr_solve_device(int N, int d, int L, double* v_dev, const trstmi_tr_options& o,
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
  T.coef = T.dots + 3 * L;
  T.deltas = T.coef + 2 * (size_t)kCoefRing * L;
  T.flag = reinterpret_cast<int*>(T.deltas + L);
  T.bad = reinterpret_cast<uint32_t*>(T.flag + L);
  const size_t small_bytes = (((size_t)L * (2 + 3 + 2 * kCoefRing + 1) * sizeof(double) +
                               (size_t)L * (sizeof(int) + sizeof(uint32_t))) + 255) & ~(size_t)255;
  T.lse = b + 9 * vec + small_bytes;
  T.x = v_dev;
  void* pinned = nullptr;
  const size_t pinned_bytes = (size_t)L * (2 * kCoefRing + 2 + 3 + 1) * sizeof(double) +
                              (size_t)L * (sizeof(int) + sizeof(uint32_t));
  if (cudaMallocHost(&pinned, pinned_bytes) != cudaSuccess) return TRSTMI_ENOMEM;
  T.h_coef = static_cast<double*>(pinned);
  T.h_out = T.h_coef + 2 * (size_t)kCoefRing * L;
  T.h_dots = T.h_out + 2 * L;
  T.h_deltas = T.h_dots + 3 * L;
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
    if ((e = cg_steihaug(T, delta, o.fd_step, radius, eps, step, o.max_cg, m, cgit, cgst,
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

}  // namespace trstmi
