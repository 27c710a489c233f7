// Projection onto previous solutions for successive right-hand sides (arXiv
// 2107.01243 §4 and Table 2: Neko starts its pressure solves from the
// projection onto a space of 20 previous solutions, after Nek5000).
//
// The space X = [x_1 .. x_l] is kept H-orthonormal in the unique-dof inner
// product, with W = H X stored beside it.  A solve of H x = b:
//   alpha = X^T b, x_bar = X alpha, r = b - W alpha     (one pass each, no matvec)
//   PCG on H d = r from d = 0 to ||b - H x|| <= tol ||b||;  x = x_bar + d
//   w = H d (one matvec); d, w H-orthogonalised against the space by
//   Gram-Schmidt applied twice, normalised by sqrt(<d, w>) and appended; a full
//   space restarts from the latest solution (H x = W alpha + w needs no matvec).
// All vectors are FP64 L-vectors; the coefficients stay on the device between
// the dot and combination kernels.
#include <cmath>
#include <memory>
#include <vector>

#include "sem_internal.cuh"
#include "reduce.cuh"
#include "krylov.cuh"

namespace sem {

constexpr int kMaxProj = 64;          // largest space
}  // namespace sem

using namespace sem;

struct sem_proj {
  sem_handle* h = nullptr;
  int m = 0, l = 0;
  std::vector<std::unique_ptr<DevBuf<double>>> X, W;
  DevBuf<const double*> xptr, wptr, one;   // device pointer arrays
  DevBuf<double> coef;                     // kMaxProj coefficients
  DevBuf<double> dots;                     // scalar results
  DevBuf<double> partials;
  DevBuf<unsigned> counter;
  DevBuf<double> xbar, r, d, hd, t1;       // scratch L-vectors
  double* pin = nullptr;                   // pinned host scalars
  ~sem_proj() {
    if (pin) cudaFreeHost(pin);
  }
};

namespace {

// <V_i, b> for i < cnt into dst (device), chunks of kDotChunk vectors
void mdot(sem_proj* pr, const double* const* V, int cnt, const double* b, double* dst,
          cudaStream_t s) {
  const int64_t n = pr->h->nL;
  for (int i0 = 0; i0 < cnt; i0 += kDotChunk) {
    const int c = std::min(kDotChunk, cnt - i0);
    k_mdot<kDotChunk><<<kRedBlocks, kRedThreads, 0, s>>>(n, V, i0, c, b, pr->h->imult.ptr, dst,
                                                         pr->partials.ptr, pr->counter.ptr);
    SEM_CHECK_LAUNCH();
  }
}

// <a, b> on the host (synchronises)
double dot_host(sem_proj* pr, const double* a, const double* b, cudaStream_t s) {
  const double* ptrs[1] = {a};
  SEM_CUDA(cudaMemcpyAsync(pr->one.ptr, ptrs, sizeof(ptrs), cudaMemcpyHostToDevice, s));
  mdot(pr, pr->one.ptr, 1, b, pr->dots.ptr, s);
  SEM_CUDA(cudaMemcpyAsync(pr->pin, pr->dots.ptr, sizeof(double), cudaMemcpyDeviceToHost, s));
  SEM_CUDA(cudaStreamSynchronize(s));
  return pr->pin[0];
}

// append (v, hv) after H-Gram-Schmidt against the space (twice); v, hv are scratch
void orthonormal_add(sem_proj* pr, double* v, double* hv, cudaStream_t s) {
  const int64_t n = pr->h->nL;
  const double d0 = dot_host(pr, v, hv, s);
  for (int pass = 0; pass < 2 && pr->l > 0; ++pass) {
    mdot(pr, pr->xptr.ptr, pr->l, hv, pr->coef.ptr, s);             // c_i = <x_i, H v>
    k_mcomb<<<lin_grid(n), 256, 0, s>>>(n, pr->xptr.ptr, pr->l, pr->coef.ptr, -1.0, v, v);
    SEM_CHECK_LAUNCH();
    k_mcomb<<<lin_grid(n), 256, 0, s>>>(n, pr->wptr.ptr, pr->l, pr->coef.ptr, -1.0, hv, hv);
    SEM_CHECK_LAUNCH();
  }
  const double nrm2 = dot_host(pr, v, hv, s);
  if (!(nrm2 > 0.0) || !(nrm2 > 1e-20 * std::fabs(d0))) return;
  const double sc = 1.0 / std::sqrt(nrm2);
  k_scale2<<<lin_grid(n), 256, 0, s>>>(n, v, hv, sc, pr->X[pr->l]->ptr, pr->W[pr->l]->ptr);
  SEM_CHECK_LAUNCH();
  ++pr->l;
}

}  // namespace

extern "C" sem_status sem_proj_create(sem_handle* h, int m, sem_proj** out) {
  return guarded("sem_proj_create", [&] {
    SEM_REQUIRE(h && out, "sem_proj_create: null argument");
    SEM_REQUIRE(m >= 0 && m <= kMaxProj, "sem_proj_create: space size must be in [0, 64]");
    SEM_REQUIRE(h->f64.G.ptr, "sem_proj_create: handle has no FP64 geometry");
    *out = nullptr;
    std::unique_ptr<sem_proj> pr(new sem_proj());
    pr->h = h;
    pr->m = m;
    const int64_t n = h->nL;
    std::vector<const double*> xp(std::max(1, m)), wp(std::max(1, m));
    for (int i = 0; i < m; ++i) {
      pr->X.emplace_back(new DevBuf<double>());
      pr->W.emplace_back(new DevBuf<double>());
      pr->X[i]->alloc(n);
      pr->W[i]->alloc(n);
      xp[i] = pr->X[i]->ptr;
      wp[i] = pr->W[i]->ptr;
    }
    pr->xptr.alloc(xp.size());
    pr->wptr.alloc(wp.size());
    pr->xptr.upload(xp.data(), xp.size(), nullptr);
    pr->wptr.upload(wp.data(), wp.size(), nullptr);
    pr->one.alloc(1);
    pr->coef.alloc(kMaxProj);
    pr->dots.alloc(kMaxProj);
    pr->partials.alloc((size_t)kDotChunk * kRedBlocks);
    pr->counter.alloc(1);
    SEM_CUDA(cudaMemset(pr->counter.ptr, 0, sizeof(unsigned)));
    pr->xbar.alloc(n);
    pr->r.alloc(n);
    pr->d.alloc(n);
    pr->hd.alloc(n);
    pr->t1.alloc(n);
    SEM_CUDA(cudaMallocHost(&pr->pin, 4 * sizeof(double)));
    SEM_CUDA(cudaDeviceSynchronize());
    *out = pr.release();
  });
}

extern "C" sem_status sem_proj_size(const sem_proj* pr, int* l) {
  return guarded("sem_proj_size", [&] {
    SEM_REQUIRE(pr && l, "sem_proj_size: null argument");
    *l = pr->l;
  });
}

extern "C" sem_status sem_proj_reset(sem_proj* pr) {
  return guarded("sem_proj_reset", [&] {
    SEM_REQUIRE(pr, "sem_proj_reset: null argument");
    pr->l = 0;
  });
}

extern "C" sem_status sem_proj_destroy(sem_proj* pr) {
  return guarded("sem_proj_destroy", [&] {
    if (!pr) return;
    cudaDeviceSynchronize();
    delete pr;
  });
}

extern "C" sem_status sem_proj_solve(sem_proj* pr, const double* b_L, double* x_L,
                                     const sem_solve_opts* opts, sem_solve_info* info) {
  sem_status inner_status = SEM_OK;
  sem_status st = guarded("sem_proj_solve", [&] {
    SEM_REQUIRE(pr && b_L && x_L, "sem_proj_solve: null argument");
    sem_solve_opts o;
    if (opts) o = *opts; else sem_solve_opts_default(&o);
    SEM_REQUIRE(o.h1_field == nullptr, "sem_proj_solve: a per-point h1 is not supported");
    sem_handle* h = pr->h;
    const int64_t n = h->nL;
    cudaStream_t s = (cudaStream_t)o.stream;
    const double bb = dot_host(pr, b_L, b_L, s);
    // x_bar and r = b - W alpha
    const int l0 = pr->l;
    if (l0 > 0) {
      mdot(pr, pr->xptr.ptr, l0, b_L, pr->coef.ptr, s);
      k_mcomb<<<lin_grid(n), 256, 0, s>>>(n, pr->xptr.ptr, l0, pr->coef.ptr, 1.0, nullptr,
                                          pr->xbar.ptr);
      SEM_CHECK_LAUNCH();
      k_mcomb<<<lin_grid(n), 256, 0, s>>>(n, pr->wptr.ptr, l0, pr->coef.ptr, -1.0, b_L,
                                          pr->r.ptr);
      SEM_CHECK_LAUNCH();
    } else {
      SEM_CUDA(cudaMemsetAsync(pr->xbar.ptr, 0, n * sizeof(double), s));
      SEM_CUDA(cudaMemcpyAsync(pr->r.ptr, b_L, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    const double rr = dot_host(pr, pr->r.ptr, pr->r.ptr, s);
    sem_solve_info in{};
    if (bb == 0.0 || rr <= o.tol * o.tol * bb) {
      SEM_CUDA(cudaMemsetAsync(pr->d.ptr, 0, n * sizeof(double), s));
      in.status = SEM_OK;
    } else {
      sem_solve_opts oi = o;
      oi.tol = o.tol * std::sqrt(bb / rr);
      oi.x0_is_zero = 1;
      const sem_status cs = sem_cg_solve(h, pr->r.ptr, pr->d.ptr, &oi, &in);
      if (cs != SEM_OK && cs != SEM_ERR_NOCONV && cs != SEM_ERR_BREAKDOWN)
        throw Error(cs, sem_last_error());
      inner_status = cs;
    }
    // x = x_bar + d;  H d;  the true residual b - H x = r - H d
    k_lin3<<<lin_grid(n), 256, 0, s>>>(n, pr->xbar.ptr, pr->d.ptr, nullptr, 1.0, x_L);
    SEM_CHECK_LAUNCH();
    launch_apply<double>(h, h->f64, pr->d.ptr, pr->hd.ptr, o.h1, o.h2, nullptr, nullptr,
                         SEM_APPLY_FULL, s);
    k_lin3<<<lin_grid(n), 256, 0, s>>>(n, pr->r.ptr, pr->hd.ptr, nullptr, -1.0, pr->t1.ptr);
    SEM_CHECK_LAUNCH();
    const double res2 = dot_host(pr, pr->t1.ptr, pr->t1.ptr, s);
    // add the correction, or restart from x when the space is full
    if (pr->m > 0) {
      if (pr->l >= pr->m) {
        // H x = W alpha + H d = (b - r) + H d, into t1; x copied to d
        k_lin3<<<lin_grid(n), 256, 0, s>>>(n, b_L, pr->r.ptr, pr->hd.ptr, -1.0, pr->t1.ptr);
        SEM_CHECK_LAUNCH();
        SEM_CUDA(cudaMemcpyAsync(pr->d.ptr, x_L, n * sizeof(double), cudaMemcpyDeviceToDevice,
                                 s));
        pr->l = 0;
        orthonormal_add(pr, pr->d.ptr, pr->t1.ptr, s);
      } else {
        orthonormal_add(pr, pr->d.ptr, pr->hd.ptr, s);
      }
    }
    SEM_CUDA(cudaStreamSynchronize(s));
    if (info) {
      info->iters = in.iters;
      info->outer_iters = in.outer_iters;
      info->rel_res = bb > 0 ? std::sqrt(res2 / bb) : 0.0;
      info->status = in.status;
    }
  });
  if (st != SEM_OK) return st;
  return inner_status;
}
