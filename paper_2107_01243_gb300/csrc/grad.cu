// Per-point derivative of lambda^T H(h1) u with respect to h1, negated:
// g = -(D^ lambda)^T G (D^ u), D^ = (d/dr, d/ds, d/dt) at each GLL point.
// H depends on h1 only through h1 G inside A^e = D^T (h1 G) D (arXiv
// 2107.01243 §2, Eq. 9), so with lambda the adjoint solution this is dL/dh1.
#include "sem_internal.cuh"

namespace sem {

template <int P>
__global__ void __launch_bounds__(P * P * 2)
grad_kernel(const double* __restrict__ u, const double* __restrict__ lam,
            const double* __restrict__ G, const double* __restrict__ Dg, double* __restrict__ gout,
            int E) {
  constexpr int P2 = P * P, P3 = P2 * P, PP = P + 1, PL = P * PP, VOL = P * PL, EPB = 2;
  __shared__ double sD[P][PP];
  __shared__ double su[EPB][VOL];
  __shared__ double sl[EPB][VOL];
  const int tid = threadIdx.x, el = threadIdx.y;
  const int i = tid % P, j = tid / P;
  for (int q = tid + el * P2; q < P2; q += P2 * EPB) sD[q / P][q % P] = Dg[q];
  __syncthreads();
  for (int e0 = blockIdx.x * EPB; e0 < E; e0 += gridDim.x * EPB) {
    const int e = e0 + el;
    const bool act = e < E;
    const size_t base = (size_t)(act ? e : 0) * P3 + tid;
    double uc[P], lc[P];
#pragma unroll
    for (int k = 0; k < P; ++k) {
      uc[k] = act ? u[base + k * P2] : 0.0;
      lc[k] = act ? lam[base + k * P2] : 0.0;
      su[el][k * PL + j * PP + i] = uc[k];
      sl[el][k * PL + j * PP + i] = lc[k];
    }
    __syncthreads();
    const double* g = G + (size_t)(act ? e : 0) * 6 * P3 + tid;
#pragma unroll
    for (int k = 0; k < P; ++k) {
      double ur = 0, us = 0, ut = 0, lr = 0, ls = 0, lt = 0;
#pragma unroll
      for (int l = 0; l < P; ++l) {
        ur += sD[i][l] * su[el][k * PL + j * PP + l];
        us += sD[j][l] * su[el][k * PL + l * PP + i];
        ut += sD[k][l] * uc[l];
        lr += sD[i][l] * sl[el][k * PL + j * PP + l];
        ls += sD[j][l] * sl[el][k * PL + l * PP + i];
        lt += sD[k][l] * lc[l];
      }
      double g11 = g[0 * P3 + k * P2], g22 = g[1 * P3 + k * P2], g33 = g[2 * P3 + k * P2];
      double g12 = g[3 * P3 + k * P2], g13 = g[4 * P3 + k * P2], g23 = g[5 * P3 + k * P2];
      double vr = g11 * ur + g12 * us + g13 * ut;
      double vs = g12 * ur + g22 * us + g23 * ut;
      double vt = g13 * ur + g23 * us + g33 * ut;
      if (act) gout[base + k * P2] = -(lr * vr + ls * vs + lt * vt);
    }
    __syncthreads();
  }
}

template <int P>
static void launch_grad_p(const sem_handle* h, const double* u, const double* lam, double* g,
                          cudaStream_t s) {
  const int E = (int)h->E;
  dim3 block(P * P, 2);
  grad_kernel<P><<<(E + 1) / 2, block, 0, s>>>(u, lam, h->f64.G.ptr, h->f64.D.ptr, g, E);
  SEM_CHECK_LAUNCH();
}

void launch_grad(const sem_handle* h, const double* u, const double* lam, double* g,
                 cudaStream_t s) {
  switch (h->P) {
    case 2: launch_grad_p<2>(h, u, lam, g, s); break;
    case 3: launch_grad_p<3>(h, u, lam, g, s); break;
    case 4: launch_grad_p<4>(h, u, lam, g, s); break;
    case 5: launch_grad_p<5>(h, u, lam, g, s); break;
    case 6: launch_grad_p<6>(h, u, lam, g, s); break;
    case 7: launch_grad_p<7>(h, u, lam, g, s); break;
    case 8: launch_grad_p<8>(h, u, lam, g, s); break;
    case 9: launch_grad_p<9>(h, u, lam, g, s); break;
    case 10: launch_grad_p<10>(h, u, lam, g, s); break;
    case 11: launch_grad_p<11>(h, u, lam, g, s); break;
    default: throw Error(SEM_ERR_ARG, "launch_grad: unsupported order");
  }
}

}  // namespace sem

using namespace sem;

extern "C" sem_status sem_helmholtz_grad(sem_handle* h, const double* u_L,
                                         const double* lambda_L, double* g_L, void* stream) {
  return guarded("sem_helmholtz_grad", [&] {
    SEM_REQUIRE(h && u_L && lambda_L && g_L, "sem_helmholtz_grad: null argument");
    launch_grad(h, u_L, lambda_L, g_L, (cudaStream_t)stream);
  });
}
