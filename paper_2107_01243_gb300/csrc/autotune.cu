// Autotuner for the element operator: for the handle's order and size it
// times every candidate tile of the FP32 Ax (global-load kernel, or the
// bulk-copy kernel with 1-3 shared-memory stages and 1 or 2 elements per
// CTA) and of the double-float FP64 Ax (1 or 2 stages) on the handle's own
// geometry, keeps the fastest in the handle, and remembers it per (order,
// precision, element-count bucket) for the process.  With SEM_AUTOTUNE_CACHE
// set to a file path the choices are also read from and appended to that
// file, so later processes skip the timing.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

#include "sem_internal.cuh"

namespace sem {

namespace {

// FP32 bulk-copy variants: (stages, elements per CTA) as in ax_tma.cu
constexpr int kTmaStages[5] = {1, 2, 3, 1, 2};
constexpr int kTmaElems[5] = {1, 1, 1, 2, 2};

struct Choice {
  int ax32_ldg, ax32_variant, df_variant;
};

std::mutex g_mu;
std::map<std::tuple<int, int>, Choice> g_cache;   // (P, log2 E bucket) -> choice
bool g_file_loaded = false;

int ebucket(int64_t E) {
  int b = 0;
  while ((1LL << (b + 1)) <= E) ++b;
  return b;
}

const char* cache_path() { return std::getenv("SEM_AUTOTUNE_CACHE"); }

void load_file_locked() {
  if (g_file_loaded) return;
  g_file_loaded = true;
  const char* path = cache_path();
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  int P, b, l, v, d;
  while (std::fscanf(f, "%d %d %d %d %d", &P, &b, &l, &v, &d) == 5) {
    // entries outside the tuner's own choices (a damaged or foreign file) are
    // skipped: the variant indexes the stage tables
    if (P < 2 || P > kMaxP || b < 0 || b > 62 || (l != 0 && l != 1) || v < 0 || v >= 5 ||
        (d != 0 && d != 1))
      continue;
    g_cache[std::make_tuple(P, b)] = Choice{l, v, d};
  }
  std::fclose(f);
}

void append_file_locked(int P, int b, const Choice& c) {
  const char* path = cache_path();
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%d %d %d %d %d\n", P, b, c.ax32_ldg, c.ax32_variant, c.df_variant);
  std::fclose(f);
}

// mean milliseconds per call of fn over reps calls (after one warm-up call)
template <class F>
float time_calls(F fn, cudaStream_t s, int reps) {
  cudaEvent_t a, b;
  SEM_CUDA(cudaEventCreate(&a));
  SEM_CUDA(cudaEventCreate(&b));
  fn();
  SEM_CUDA(cudaEventRecord(a, s));
  for (int r = 0; r < reps; ++r) fn();
  SEM_CUDA(cudaEventRecord(b, s));
  SEM_CUDA(cudaEventSynchronize(b));
  float ms = 0.0f;
  SEM_CUDA(cudaEventElapsedTime(&ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms / reps;
}

}  // namespace

}  // namespace sem

using namespace sem;

extern "C" sem_status sem_autotune(sem_handle* h, void* stream, sem_tuning* out) {
  return guarded("sem_autotune", [&] {
    SEM_REQUIRE(h, "sem_autotune: null handle");
    cudaStream_t s = (cudaStream_t)stream;
    const int b = ebucket(h->E);
    const auto key = std::make_tuple(h->P, b);
    std::lock_guard<std::mutex> lock(g_mu);
    load_file_locked();
    sem_tuning t{};
    t.ax32_ms = -1.0;
    t.ax64_ms = -1.0;
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      h->tune.ax32_ldg = it->second.ax32_ldg;
      h->tune.ax32_variant = it->second.ax32_variant;
      h->tune.df_variant = it->second.df_variant;
      t.from_cache = 1;
    } else {
      const int64_t n = h->nL;
      const int reps = h->nL > (1 << 22) ? 3 : 10;
      Choice best{h->tune.ax32_ldg, h->tune.ax32_variant, h->tune.df_variant};
      if (h->f32.G.ptr) {
        DevBuf<float> u, w;
        u.alloc(n);
        w.alloc(n);
        // non-zero data (zeros take shortcuts in some kernels): every byte 0x3F
        SEM_CUDA(cudaMemsetAsync(u.ptr, 0x3F, n * sizeof(float), s));
        float bt = 1e30f;
        auto run32 = [&]() {
          launch_ax<float>(h, h->f32, u.ptr, w.ptr, 1.0f, 0.0f, nullptr, nullptr, s);
        };
        h->tune.ax32_ldg = 1;
        float ms = time_calls(run32, s, reps);
        if (ms < bt) { bt = ms; best.ax32_ldg = 1; }
        if (tma_ax_supported<float>(h, u.ptr, w.ptr, nullptr)) {
          h->tune.ax32_ldg = 0;
          for (int v = 0; v < 5; ++v) {
            h->tune.ax32_variant = v;
            ms = time_calls(run32, s, reps);
            if (ms < bt) { bt = ms; best.ax32_ldg = 0; best.ax32_variant = v; }
          }
        }
        t.ax32_ms = bt;
      }
      if (h->gdf.ptr) {
        DevBuf<double> u, w;
        u.alloc(n);
        w.alloc(n);
        SEM_CUDA(cudaMemsetAsync(u.ptr, 0x3F, n * sizeof(double), s));
        SEM_REQUIRE(df_ax_supported(h, u.ptr, w.ptr, nullptr), "sem_autotune: double-float Ax");
        float bt = 1e30f;
        for (int v = 0; v < 2; ++v) {
          h->tune.df_variant = v;
          const float ms = time_calls([&]() { launch_ax_df(h, u.ptr, w.ptr, 1.0, 0.0, nullptr, s); },
                                      s, reps);
          if (ms < bt) { bt = ms; best.df_variant = v; }
        }
        t.ax64_ms = bt;
      }
      h->tune.ax32_ldg = best.ax32_ldg;
      h->tune.ax32_variant = best.ax32_variant;
      h->tune.df_variant = best.df_variant;
      g_cache[key] = best;
      append_file_locked(h->P, b, best);
      SEM_CUDA(cudaStreamSynchronize(s));
    }
    h->tune.tuned = 1;
    t.ax32_kernel = h->tune.ax32_ldg ? 1 : 0;
    t.ax32_stages = kTmaStages[h->tune.ax32_variant];
    t.ax32_elems_per_cta = kTmaElems[h->tune.ax32_variant];
    t.f64_stages = h->tune.df_variant + 1;
    if (out) *out = t;
  });
}

extern "C" sem_status sem_set_tuning(sem_handle* h, const sem_tuning* t) {
  return guarded("sem_set_tuning", [&] {
    SEM_REQUIRE(h && t, "sem_set_tuning: null argument");
    SEM_REQUIRE(t->ax32_kernel == 0 || t->ax32_kernel == 1, "sem_set_tuning: bad ax32_kernel");
    SEM_REQUIRE(t->f64_stages == 1 || t->f64_stages == 2, "sem_set_tuning: bad f64_stages");
    int v = -1;
    for (int q = 0; q < 5; ++q)
      if (kTmaStages[q] == t->ax32_stages && kTmaElems[q] == t->ax32_elems_per_cta) v = q;
    SEM_REQUIRE(v >= 0, "sem_set_tuning: no such (stages, elements per CTA) variant");
    h->tune.ax32_ldg = t->ax32_kernel;
    h->tune.ax32_variant = v;
    h->tune.df_variant = t->f64_stages - 1;
  });
}
