// Gather-scatter QQ^T with the Dirichlet mask (arXiv 2107.01243 §2, Eq. 10;
// §3.2).  Local points that share a global number are grouped in segments
// (local indices ascending inside a segment, segments ordered by global
// number); one thread sums a segment in that order and writes the sum back to
// every copy, so the result does not depend on scheduling.  Points owned by
// one element only are untouched; Dirichlet points are listed separately and
// zeroed when the mask is applied.
#include "sem_internal.cuh"

namespace sem {

template <class T>
__global__ void dssum_kernel(T* __restrict__ w, const int* __restrict__ seg_ptr,
                             const int* __restrict__ seg_idx, int nseg,
                             const int* __restrict__ masked, int nmasked,
                             const CGState* __restrict__ st) {
  if (st && st->done) return;
  const int total = nseg + nmasked;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    if (t < nseg) {
      const int a = seg_ptr[t], b = seg_ptr[t + 1];
      T s = w[seg_idx[a]];
      for (int q = a + 1; q < b; ++q) s += w[seg_idx[q]];
      for (int q = a; q < b; ++q) w[seg_idx[q]] = s;
    } else {
      w[masked[t - nseg]] = T(0);
    }
  }
}

template <class T>
void launch_dssum(const sem_handle* h, T* w, bool apply_mask, const CGState* st, cudaStream_t s) {
  if (h->dssum_kernel == SEM_DSSUM_BOX) {
    launch_dssum_box<T>(h, w, apply_mask, st, s);
    return;
  }
  const int nseg = (int)(apply_mask ? h->nseg_free : h->nseg_all);
  const int nm = apply_mask ? (int)h->nmasked : 0;
  const int total = nseg + nm;
  if (total == 0) return;
  int blocks = std::min((total + 255) / 256, 32 * sem_num_sms());
  dssum_kernel<T><<<blocks, 256, 0, s>>>(w, h->seg_ptr.ptr, h->seg_idx.ptr, nseg,
                                         h->masked_idx.ptr, nm, st);
  SEM_CHECK_LAUNCH();
}

template void launch_dssum<double>(const sem_handle*, double*, bool, const CGState*, cudaStream_t);
template void launch_dssum<float>(const sem_handle*, float*, bool, const CGState*, cudaStream_t);

}  // namespace sem

using namespace sem;

extern "C" sem_status sem_dssum(sem_handle* h, void* w_L, int apply_mask, int dtype,
                                void* stream) {
  return guarded("sem_dssum", [&] {
    SEM_REQUIRE(h && w_L, "sem_dssum: null handle or vector");
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == SEM_F64) launch_dssum<double>(h, (double*)w_L, apply_mask != 0, nullptr, s);
    else if (dtype == SEM_F32) launch_dssum<float>(h, (float*)w_L, apply_mask != 0, nullptr, s);
    else throw Error(SEM_ERR_ARG, "sem_dssum: bad dtype");
  });
}

extern "C" sem_status sem_set_dssum_kernel(sem_handle* h, int kind) {
  return guarded("sem_set_dssum_kernel", [&] {
    SEM_REQUIRE(h, "sem_set_dssum_kernel: null handle");
    SEM_REQUIRE(kind == SEM_DSSUM_BOX || kind == SEM_DSSUM_SEGMENTS,
                "sem_set_dssum_kernel: unknown kind");
    if (kind == SEM_DSSUM_SEGMENTS) sem_build_segments(h, nullptr);
    h->dssum_kernel = kind;
  });
}
