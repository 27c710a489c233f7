// The FP32 operator on global (unique-dof) vectors, w_g = mask Q^T (h1 A_L +
// h2 B_L) Q u_g (arXiv 2107.01243 §2, Eq. 9-10, with the local-to-global map
// Q of Eq. 10 applied inside the element kernel), for the FP32 inner solves
// of the mixed-precision solver, and the conversions between L-vectors and
// global vectors.
//
// On the box the global numbering is the lattice g = ix + gx (iy + gy iz), so
// an element gathers its P^3 values as P^2 rows of P consecutive floats of
// the lattice (the faces it shares are read again, from L2, by its
// neighbours), and assembles its output directly: points inside the element
// belong to it alone and are stored, points on its faces are added with
// atomics (reductions in L2), Dirichlet points are skipped.  Global vectors
// hold about (N/(N+1))^3 of the local points (0.67 at N = 7), so each CG
// vector pass moves a third fewer bytes, and no gather-scatter pass is left.
// The order of the atomic additions varies, so FP32 results may differ in
// the last bits from run to run; the FP64 refinement around the inner solve
// is unaffected.
#include <cmath>

#include "sem_internal.cuh"
#include "tma.cuh"
#include "ax_tile.cuh"
#include "reduce.cuh"
#include "cg_state.cuh"

namespace sem {

struct GBox {
  int nelx, nely, nelz, faces;
  int gx;             // lattice extent in x
  long long sk;       // lattice stride in z: gx gy
  FastDiv dnx, dny;   // division by nelx, nely
};

// box position of element e and the lattice index of its point (0, 0, 0)
__device__ __forceinline__ long long elem_origin(int e, const GBox& b, int N, int& ex, int& ey,
                                                 int& ez) {
  const uint32_t r = b.dnx.div((uint32_t)e);
  ex = e - (int)r * b.nelx;
  const uint32_t q = b.dny.div(r);
  ey = (int)(r - q * (uint32_t)b.nely);
  ez = (int)q;
  return (long long)(ex * N) + (long long)b.gx * (ey * N) + b.sk * (long long)(ez * N);
}

// Dirichlet face bits of element (ex, ey, ez) in the point-flag layout below
__device__ __forceinline__ unsigned dirichlet_bits(const GBox& b, int ex, int ey, int ez) {
  if (!b.faces) return 0u;
  return ((b.faces & SEM_FACE_XMIN) && ex == 0 ? 4u : 0u) |
         ((b.faces & SEM_FACE_XMAX) && ex == b.nelx - 1 ? 8u : 0u) |
         ((b.faces & SEM_FACE_YMIN) && ey == 0 ? 16u : 0u) |
         ((b.faces & SEM_FACE_YMAX) && ey == b.nely - 1 ? 32u : 0u) |
         ((b.faces & SEM_FACE_ZMIN) && ez == 0 ? 64u : 0u) |
         ((b.faces & SEM_FACE_ZMAX) && ez == b.nelz - 1 ? 128u : 0u);
}

// A persistent CTA of P x P threads walks elements blockIdx.x + m gridDim.x.
// Thread 0 keeps STAGES elements' geometric factors (and B) in flight by bulk
// copies on mbarriers (a stage is refilled once the forward phase is done); every thread gathers its own k-column of the next
// element's u into a second shared buffer by cp.async while the current one
// is computed.  w must hold zeros at every unmasked point on element faces.
// pwst (P = 8): <p, H p> and alpha from the local products, p = u (the sum
// over local points of u_L (H_L u_L), equal to the global product because u
// is zero on Dirichlet points).
template <int P, int STAGES>
__global__ void __launch_bounds__(P * P)
ax_glob_kernel(const float* __restrict__ u, float* __restrict__ w, const float* __restrict__ G,
               const float* __restrict__ B, float h1, float h2, DMat<P, float> D, int E, GBox bx,
               const CGState* __restrict__ st, CGState* __restrict__ pwst,
               double* __restrict__ partials, int* __restrict__ err, uint64_t timeout_ns) {
  constexpr int P2 = P * P, P3 = P2 * P, N = P - 1;
  constexpr uint32_t FB = P3 * sizeof(float);
  if (st && st->done) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  float* stage0 = reinterpret_cast<float*>(smem_raw + 128);
  const bool helm = h2 != 0.0f;
  const int nf = 6 + (helm ? 1 : 0);
  const int SE = nf * P3;
  float* su = stage0 + STAGES * SE;        // [2][P3]: gathered u, double-buffered
  float* sT = su + 2 * P3;
  float* swr = su + 3 * P3;
  float* swsT = su + 4 * P3;
  const int tid = threadIdx.x;
  auto Dm = [&](int r, int c) { return D.d[r * P + c]; };
  TileThread<P, float> t;
  t.init(tid, Dm);
  const long long toff = t.i + (long long)bx.gx * t.j;    // this thread's (i, j, 0)
  auto gather = [&](int e, float* dst) {
    int ex, ey, ez;
    const float* src = u + elem_origin(e, bx, N, ex, ey, ez) + toff;
#pragma unroll
    for (int k = 0; k < P; ++k) cp_async4(dst + k * P2 + t.lt, src + bx.sk * k);
  };
  auto issue = [&](int e, int s) {
    float* dst = stage0 + s * SE;
    const uint64_t pol = l2_policy_evict_first();   // G and B are read once
    mbar_arrive_expect_tx(&bar[s], (uint32_t)nf * FB);
    bulk_g2s_hint(dst, G + (size_t)e * 6 * P3, 6 * FB, &bar[s], pol);
    if (helm) bulk_g2s_hint(dst + 6 * P3, B + (size_t)e * P3, FB, &bar[s], pol);
  };
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < STAGES; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  const int Gs = gridDim.x;
  int issued = 0;
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < STAGES; ++s) {
      const int e = blockIdx.x + s * Gs;
      if (e < E) {
        issue(e, s);
        ++issued;
      }
    }
  }
  if (blockIdx.x < E) gather(blockIdx.x, su);
  cp_async_commit();
  float pw_s = 0.0f, pw_c = 0.0f;          // Kahan-compensated <p, H p>
  const bool fi = t.i == 0 || t.i == N, fj = t.j == 0 || t.j == N;
  const unsigned pij = (t.i == 0 ? 4u : 0u) | (t.i == N ? 8u : 0u) | (t.j == 0 ? 16u : 0u) |
                       (t.j == N ? 32u : 0u);
  int n = 0;
  for (int e = blockIdx.x; e < E; e += Gs, ++n) {
    const int s = n % STAGES;
    const bool ok = mbar_wait_bounded(&bar[s], (uint32_t)(n / STAGES) & 1u, err, timeout_ns);
    // the other buffer was last read before the previous iteration's second barrier
    const float* cu = su + (n & 1) * P3;
    if (e + Gs < E) gather(e + Gs, su + ((n + 1) & 1) * P3);
    cp_async_commit();
    cp_async_wait<1>();                    // this thread's copies of element e landed
    float uc[P], bk[P], ck[P], wt[P];
    const float* sg = stage0 + s * SE;
#pragma unroll
    for (int k = 0; k < P; ++k) {
      uc[k] = cu[k * P2 + t.lt];
      sT[k * P2 + t.tpos] = uc[k];
      ck[k] = h1;
      bk[k] = helm ? sg[6 * P3 + k * P2 + t.lt] : 0.0f;
    }
    if (__syncthreads_or(!ok)) {
      // a copy never completed: wait (bounded) for what is in flight, then leave
      cp_async_wait<0>();
      if (tid == 0)
        for (int nn = n; nn < issued; ++nn)
          mbar_wait_bounded(&bar[nn % STAGES], (uint32_t)(nn / STAGES) & 1u, err, timeout_ns);
      break;                               // the reduction below still counts this CTA
    }
    tile_forward<P, float>(t, cu, sT, sg, uc, ck, swr, swsT, wt, Dm);
    __syncthreads();
    if (tid == 0) {                        // stage s consumed
      const int en = e + STAGES * Gs;
      if (en < E) {
        fence_proxy_async_smem();
        issue(en, s);
        ++issued;
      }
    }
    int ex, ey, ez;
    float* we = w + elem_origin(e, bx, N, ex, ey, ez) + toff;
    const unsigned fl = dirichlet_bits(bx, ex, ey, ez);
    tile_backward<P, float>(t, swr, swsT, wt, uc, bk, h2, helm, Dm, [&](int k, float v) {
      if (pwst) {
        const float y = __fsub_rn(__fmul_rn(uc[k], v), pw_c);
        const float tt = __fadd_rn(pw_s, y);
        pw_c = __fsub_rn(__fsub_rn(tt, pw_s), y);
        pw_s = tt;
      }
      const unsigned pf = pij | (k == 0 ? 64u : 0u) | (k == N ? 128u : 0u);
      if (pf & fl) return;                 // Dirichlet point: stays zero
      float* dst = we + bx.sk * k;
      if (fi || fj || k == 0 || k == N)
        red_add(dst, v);                   // shared with neighbours
      else
        *dst = v;                          // interior: this element's alone
    });
  }
  cp_async_wait<0>();
  if constexpr (P2 % 32 == 0) {
    if (pwst) {
      double v[1] = {(double)pw_s - (double)pw_c};
      double tot[1];
      if (grid_sum<1>(v, partials, &pwst->counter, tot) && threadIdx.x == 0) {
        st_after_pw(pwst, tot[0]);
      }
    }
  }
}

// one stage of geometric factors: 24.7 KB of shared memory at P = 8, eight
// CTAs per SM (two stages: six CTAs, 16% slower at 48^3 elements, N = 7)
constexpr int kGlobStages = 1;

template <int P>
static size_t glob_smem_bytes(bool helm) {
  const size_t P3 = (size_t)P * P * P;
  return 128 + (kGlobStages * (6 + (helm ? 1 : 0)) + 5) * P3 * sizeof(float);
}

static GBox make_gbox(const sem_handle* h) {
  GBox b;
  b.nelx = h->nelx;
  b.nely = h->nely;
  b.nelz = h->nelz;
  b.faces = h->faces;
  b.gx = h->N * h->nelx + 1;
  b.sk = (long long)b.gx * (h->N * h->nely + 1);
  b.dnx = FastDiv((uint32_t)h->nelx);
  b.dny = FastDiv((uint32_t)h->nely);
  return b;
}

template <int P>
static void launch_glob_p(const sem_handle* h, const float* u, float* w, float h1, float h2,
                          const CGState* st, CGState* pwst, cudaStream_t s) {
  const bool helm = h2 != 0.0f;
  auto kern = ax_glob_kernel<P, kGlobStages>;
  static bool configured = false;
  static int occ[2] = {0, 0};
  if (!configured) {
    SEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)glob_smem_bytes<P>(true)));
    configured = true;
  }
  const size_t smem = glob_smem_bytes<P>(helm);
  int& o = occ[helm ? 1 : 0];
  if (!o) {
    SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, P * P, smem));
    if (o < 1) o = 1;
  }
  DMat<P, float> D;
  for (int a = 0; a < P * P; ++a) D.d[a] = (float)h->Dh[a];
  const int E = (int)h->E;
  int grid = (int)std::min<int64_t>(E, (int64_t)o * sem_num_sms());
  if (pwst) grid = std::min(grid, kFusedPartials);
  if (grid < 1) grid = 1;
  kern<<<grid, P * P, smem, s>>>(u, w, h->f32.G.ptr, h->f32.B.ptr, h1, h2, D, E, make_gbox(h), st,
                                 pwst, h->partials.ptr + 4 * kRedBlocks, h->dev_err.ptr,
                                 kWaitTimeoutNs);
  SEM_CHECK_LAUNCH();
}

bool glob_supported(const sem_handle* h) {
  const int P = h->P;
  return h->f32.G.ptr && (P == 2 || P == 4 || P == 6 || P == 8 || P == 10) && h->E > 0 &&
         h->nL < (1LL << 31);
}

int64_t glob_padded(const sem_handle* h) { return (h->nG + 3) / 4 * 4; }

bool launch_apply_global(const sem_handle* h, const float* u, float* w, float h1, float h2,
                         const CGState* st, CGState* pwst, cudaStream_t s) {
  switch (h->P) {
    case 2: launch_glob_p<2>(h, u, w, h1, h2, st, nullptr, s); return false;
    case 4: launch_glob_p<4>(h, u, w, h1, h2, st, nullptr, s); return false;
    case 6: launch_glob_p<6>(h, u, w, h1, h2, st, nullptr, s); return false;
    case 8: launch_glob_p<8>(h, u, w, h1, h2, st, pwst, s); return pwst != nullptr;
    case 10: launch_glob_p<10>(h, u, w, h1, h2, st, nullptr, s); return false;
    default: throw Error(SEM_ERR_ARG, "apply_global: unsupported order");
  }
}

// ---------------------------------------------------------------- conversions
// Thread per global point g = ix + gx (iy + gy iz): reads the copy of g in
// element (ex, ey, ez) = (min(ix / N, nelx - 1), likewise y, z); the input is
// continuous, so every copy holds the same value.
template <class Tin>
__global__ void k_to_global(int64_t nG, const Tin* __restrict__ in, float* __restrict__ out,
                            int N, int P, int nelx, int nely, int nelz, FastDiv dgx, FastDiv dgy,
                            FastDiv dN, double scale) {
  const long long P3 = (long long)P * P * P;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nG;
       g += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t r = dgx.div((uint32_t)g);
    const int ix = (int)((uint32_t)g - r * dgx.d);
    const uint32_t izu = dgy.div(r);
    const int iy = (int)(r - izu * dgy.d), iz = (int)izu;
    const int ex = min((int)dN.div((uint32_t)ix), nelx - 1);
    const int ey = min((int)dN.div((uint32_t)iy), nely - 1);
    const int ez = min((int)dN.div((uint32_t)iz), nelz - 1);
    const int i = ix - ex * N, j = iy - ey * N, k = iz - ez * N;
    const long long e = ex + (long long)nelx * (ey + (long long)nely * ez);
    out[g] = (float)((double)in[e * P3 + ((long long)k * P + j) * P + i] * scale);
  }
}

// x_L += d_g[g(L)] at every local point
__global__ void k_add_from_global(int64_t nL, double* __restrict__ x, const float* __restrict__ d,
                                  int N, int P, int nelx, int nely, int gx, int gy, FastDiv dP3,
                                  FastDiv dP, FastDiv dnx, FastDiv dny, double scale) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nL;
       q += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t qq = (uint32_t)q;
    const uint32_t e = dP3.div(qq);
    const uint32_t lq = qq - e * dP3.d;
    const uint32_t r1 = dP.div(lq);
    const uint32_t i = lq - r1 * (uint32_t)P;
    const uint32_t k = dP.div(r1);
    const uint32_t j = r1 - k * (uint32_t)P;
    const uint32_t re = dnx.div(e);
    const uint32_t ex = e - re * (uint32_t)nelx;
    const uint32_t ez = dny.div(re);
    const uint32_t ey = re - ez * (uint32_t)nely;
    const long long g = (long long)(ex * N + i) +
                        (long long)gx * ((long long)(ey * N + j) + (long long)gy * (ez * N + k));
    x[q] += (double)d[g] * scale;
  }
}

static int conv_grid(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8 * sem_num_sms()));
}

template <class Tin>
void to_global(const sem_handle* h, const Tin* in, float* out, cudaStream_t s, double scale) {
  const int N = h->N;
  k_to_global<Tin><<<conv_grid(h->nG), 256, 0, s>>>(
      h->nG, in, out, N, h->P, h->nelx, h->nely, h->nelz, FastDiv((uint32_t)(N * h->nelx + 1)),
      FastDiv((uint32_t)(N * h->nely + 1)), FastDiv((uint32_t)(N > 0 ? N : 1)), scale);
  SEM_CHECK_LAUNCH();
}
template void to_global<float>(const sem_handle*, const float*, float*, cudaStream_t, double);
template void to_global<double>(const sem_handle*, const double*, float*, cudaStream_t, double);

void add_from_global(const sem_handle* h, double* x, const float* d, cudaStream_t s,
                     double scale) {
  k_add_from_global<<<conv_grid(h->nL), 256, 0, s>>>(
      h->nL, x, d, h->N, h->P, h->nelx, h->nely, h->N * h->nelx + 1, h->N * h->nely + 1,
      FastDiv((uint32_t)h->P3), FastDiv((uint32_t)h->P), FastDiv((uint32_t)h->nelx),
      FastDiv((uint32_t)h->nely), scale);
  SEM_CHECK_LAUNCH();
}

}  // namespace sem

using namespace sem;

extern "C" sem_status sem_apply_global(sem_handle* h, const void* u_g, void* w_g, double h1,
                                       double h2, int dtype, void* stream) {
  return guarded("sem_apply_global", [&] {
    SEM_REQUIRE(h && u_g && w_g, "sem_apply_global: null argument");
    SEM_REQUIRE(u_g != w_g, "sem_apply_global: u and w must not alias");
    SEM_REQUIRE(dtype == SEM_F32, "sem_apply_global: FP32 only");
    SEM_REQUIRE(glob_supported(h), "sem_apply_global: needs FP32 geometry, an odd order N "
                                   "and fewer than 2^31 local points");
    const cudaStream_t s = (cudaStream_t)stream;
    SEM_CUDA(cudaMemsetAsync(w_g, 0, h->nG * sizeof(float), s));
    launch_apply_global(h, (const float*)u_g, (float*)w_g, (float)h1, (float)h2, nullptr, nullptr,
                        s);
  });
}

extern "C" sem_status sem_to_global(sem_handle* h, const void* in_L, void* out_g, int dtype,
                                    void* stream) {
  return guarded("sem_to_global", [&] {
    SEM_REQUIRE(h && in_L && out_g, "sem_to_global: null argument");
    SEM_REQUIRE(dtype == SEM_F32 || dtype == SEM_F64, "sem_to_global: dtype");
    SEM_REQUIRE(h->nL < (1LL << 31), "sem_to_global: needs fewer than 2^31 local points");
    if (dtype == SEM_F32)
      to_global<float>(h, (const float*)in_L, (float*)out_g, (cudaStream_t)stream);
    else
      to_global<double>(h, (const double*)in_L, (float*)out_g, (cudaStream_t)stream);
  });
}
