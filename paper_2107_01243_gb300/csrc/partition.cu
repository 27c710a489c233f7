// Building blocks for an element partition across processes and for Krylov
// loops driven by the caller (arXiv 2107.01243 §3.2, Algorithm 1).
//
// Neko splits the elements over MPI ranks; the gather-scatter sums a shared
// point's copies inside the rank, then exchanges the partial sums of the
// points on the rank's interfaces and adds what the neighbours sent, and the
// Krylov dots end in one global reduction each.  Here a rank owns a sub-box of
// the element box with its own handle (sem_setup on the sub-box, Dirichlet
// faces only where the sub-box touches the global boundary), and the
// exchange and reductions are the caller's (the Python layer runs them over
// torch.distributed).  This file gives the device side:
//   * sem_gather / sem_scatter_add: interface values to and from contiguous
//     buffers by index lists (the caller's host logic builds them from the
//     box numbering);
//   * sem_set_multiplicity: the dots' 1/multiplicity replaced by the global
//     one (copies on other ranks included), so that sem_dot gives each rank's
//     share of the unique-dof inner product;
//   * sem_jacobi_diag / sem_jacobi_invert: the rank's assembled diagonal
//     and, after the interface sum, the masked inverse;
//   * sem_cg_update / sem_cg_direction: the PCG vector updates with the
//     rank's shares of <r, z> and <r, r>.
// Index arguments are bounds-checked in the kernels: an index outside the
// vector is skipped and SEM_ERR_ARG is recorded in the handle's device error
// word (reported by sem_sync).
#include "sem_internal.cuh"
#include "reduce.cuh"

namespace sem {

__global__ void k_gather(int64_t n, int64_t nsrc, const double* __restrict__ src,
                         const int64_t* __restrict__ idx, double* __restrict__ dst,
                         int* __restrict__ err) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = idx[t];
    if ((uint64_t)q < (uint64_t)nsrc) {
      dst[t] = src[q];
    } else {
      dst[t] = 0.0;
      atomicExch(err, (int)SEM_ERR_ARG);
    }
  }
}

// dst[idx[t]] += src[pos[t]]; the idx[t] are distinct, so no two threads add
// to one entry
__global__ void k_scatter_add(int64_t n, int64_t ndst, int64_t nsrc, double* __restrict__ dst,
                              const int64_t* __restrict__ idx, const int64_t* __restrict__ pos,
                              const double* __restrict__ src, int* __restrict__ err) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = idx[t], m = pos[t];
    if ((uint64_t)q < (uint64_t)ndst && (uint64_t)m < (uint64_t)nsrc)
      dst[q] += src[m];
    else
      atomicExch(err, (int)SEM_ERR_ARG);
  }
}

// 1/mult as float (exact for the powers of two a box produces); an entry
// that is not a positive multiplicity records an error and keeps 1
__global__ void k_set_imult(int64_t n, const double* __restrict__ mult, float* __restrict__ imult,
                            int* __restrict__ err) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    const double m = mult[q];
    if (m >= 1.0) {
      imult[q] = (float)(1.0 / m);
    } else {
      imult[q] = 1.0f;
      atomicExch(err, (int)SEM_ERR_ARG);
    }
  }
}

__global__ void k_jacobi_invert(int64_t n, const double* __restrict__ d,
                                const uint8_t* __restrict__ mask, double* __restrict__ dinv) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    dinv[q] = mask[q] ? 1.0 / d[q] : 0.0;
}

// x += alpha p, r -= alpha w, z = dinv r; the shares of <r, z> and <r, r>
// (weighted by 1/mult) into dots[0], dots[1]
__global__ void __launch_bounds__(kRedThreads)
k_cg_update(int64_t n, double alpha, const double* __restrict__ p, const double* __restrict__ w,
            double* __restrict__ x, double* __restrict__ r, const double* __restrict__ dinv,
            double* __restrict__ z, const float* __restrict__ imult, double* __restrict__ dots,
            double* __restrict__ partials, unsigned int* __restrict__ counter) {
  double v[2] = {0.0, 0.0};
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    x[q] += alpha * p[q];
    const double rq = r[q] - alpha * w[q];
    r[q] = rq;
    const double zq = dinv[q] * rq;
    z[q] = zq;
    const double im = (double)imult[q];
    v[0] += rq * zq * im;
    v[1] += rq * rq * im;
  }
  double tot[2];
  if (grid_sum<2>(v, partials, counter, tot) && threadIdx.x == 0) {
    dots[0] = tot[0];
    dots[1] = tot[1];
  }
}

__global__ void k_cg_direction(int64_t n, double beta, const double* __restrict__ z,
                               double* __restrict__ p) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    p[q] = z[q] + beta * p[q];
}

static int part_grid(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8LL * sem_num_sms()));
}

}  // namespace sem

using namespace sem;

extern "C" sem_status sem_gather(sem_handle* h, const double* src_L, const int64_t* idx,
                                 int64_t n, double* dst, void* stream) {
  return guarded("sem_gather", [&] {
    SEM_REQUIRE(h, "sem_gather: null handle");
    SEM_REQUIRE(n >= 0, "sem_gather: negative count");
    if (n == 0) return;
    SEM_REQUIRE(src_L && idx && dst, "sem_gather: null argument");
    k_gather<<<part_grid(n), 256, 0, (cudaStream_t)stream>>>(n, h->nL, src_L, idx, dst,
                                                             h->dev_err.ptr);
    SEM_CHECK_LAUNCH();
  });
}

extern "C" sem_status sem_scatter_add(sem_handle* h, double* dst_L, const int64_t* idx,
                                      const int64_t* pos, int64_t n, const double* src,
                                      int64_t n_src, void* stream) {
  return guarded("sem_scatter_add", [&] {
    SEM_REQUIRE(h, "sem_scatter_add: null handle");
    SEM_REQUIRE(n >= 0 && n_src >= 0, "sem_scatter_add: negative count");
    if (n == 0) return;
    SEM_REQUIRE(dst_L && idx && pos && src, "sem_scatter_add: null argument");
    k_scatter_add<<<part_grid(n), 256, 0, (cudaStream_t)stream>>>(n, h->nL, n_src, dst_L, idx,
                                                                  pos, src, h->dev_err.ptr);
    SEM_CHECK_LAUNCH();
  });
}

extern "C" sem_status sem_set_multiplicity(sem_handle* h, const double* mult_L, void* stream) {
  return guarded("sem_set_multiplicity", [&] {
    SEM_REQUIRE(h && mult_L, "sem_set_multiplicity: null argument");
    k_set_imult<<<part_grid(h->nL), 256, 0, (cudaStream_t)stream>>>(h->nL, mult_L, h->imult.ptr,
                                                                    h->dev_err.ptr);
    SEM_CHECK_LAUNCH();
    h->dinv_valid = 0;                 // the solvers' dinv / mult folds depend on it
  });
}

extern "C" sem_status sem_jacobi_diag(sem_handle* h, double h1, double h2, double* d_L,
                                      void* stream) {
  return guarded("sem_jacobi_diag", [&] {
    SEM_REQUIRE(h && d_L, "sem_jacobi_diag: null argument");
    cudaStream_t s = (cudaStream_t)stream;
    launch_local_diag<double>(h, h->f64, d_L, h1, h2, nullptr, s);
    launch_dssum<double>(h, d_L, false, nullptr, s);
  });
}

extern "C" sem_status sem_jacobi_invert(sem_handle* h, const double* d_L, double* dinv_L,
                                        void* stream) {
  return guarded("sem_jacobi_invert", [&] {
    SEM_REQUIRE(h && d_L && dinv_L, "sem_jacobi_invert: null argument");
    k_jacobi_invert<<<part_grid(h->nL), 256, 0, (cudaStream_t)stream>>>(h->nL, d_L, h->mask.ptr,
                                                                        dinv_L);
    SEM_CHECK_LAUNCH();
  });
}

extern "C" sem_status sem_cg_update(sem_handle* h, double alpha, const double* p, const double* w,
                                    double* x, double* r, const double* dinv, double* z,
                                    double* dots, void* stream) {
  return guarded("sem_cg_update", [&] {
    SEM_REQUIRE(h && p && w && x && r && dinv && z && dots, "sem_cg_update: null argument");
    k_cg_update<<<kRedBlocks, kRedThreads, 0, (cudaStream_t)stream>>>(
        h->nL, alpha, p, w, x, r, dinv, z, h->imult.ptr, dots,
        h->partials.ptr + 4 * kRedBlocks + kFusedPartials, &h->state.ptr[3].counter);
    SEM_CHECK_LAUNCH();
  });
}

extern "C" sem_status sem_cg_direction(sem_handle* h, double beta, const double* z, double* p,
                                       void* stream) {
  return guarded("sem_cg_direction", [&] {
    SEM_REQUIRE(h && z && p, "sem_cg_direction: null argument");
    k_cg_direction<<<part_grid(h->nL), 256, 0, (cudaStream_t)stream>>>(h->nL, beta, z, p);
    SEM_CHECK_LAUNCH();
  });
}
