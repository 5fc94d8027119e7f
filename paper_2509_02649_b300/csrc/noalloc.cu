// fk_type1_noalloc: the type-1 transform for callers that cannot allocate device
// memory.
//
// fk_type1 takes its scratch (the upsampled grid, twiddles, correction factors,
// the 2-D row-transform intermediate, an error flag) from cudaMallocAsync.  Some
// callers cannot allocate at call time: a process whose device memory is wholly
// reserved by its own pool allocator, or a service whose policy forbids device
// allocation after start-up.  This variant takes all of that scratch from one
// file-scope device array of FK_NOALLOC_SCRATCH_BYTES instead.  Every GPU that
// loads the library holds that array until the process exits.
//
// In host code the array's name is only a host-side stand-in, not a device
// address, so the first call on each device looks up the real address with
// cudaGetSymbolAddress (with that device current) and caches it; that first call
// should come before any stream capture.  All calls share the array and it keeps
// the last call's contents: the grid and the flag word are cleared on every call,
// and calls whose work overlaps on the GPU (different streams, or host threads
// calling concurrently) race on it.  The spreading step is the atomic form for
// both precisions.  The paper has no counterpart to this entry point.
#include "fk_internal.cuh"

#include <mutex>

namespace fk {
namespace {

constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[FK_NOALLOC_SCRATCH_BYTES];

std::mutex g_mutex;
void* g_addr[MAX_DEVICES] = {nullptr};

fk_status scratch_address(void** out) {
  int dev = 0;
  FK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES) return set_error(FK_EINVAL, "device %d beyond the supported %d", dev, MAX_DEVICES);
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return set_error(FK_ECUDA, "cudaGetSymbolAddress of the no-allocation scratch failed: %s", cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return FK_OK;
}

size_t align256(size_t v) { return (v + 255) & ~static_cast<size_t>(255); }

}  // namespace
}  // namespace fk

using namespace fk;

extern "C" fk_status fk_type1_noalloc(int d, int64_t n, const void* x, const void* c, int n_ch, int kmax, double eps,
                                      int precision, double* out, void* stream) {
  clear_error();
  if (d < 1 || d > 2) return set_error(FK_EINVAL, "d = %d: transforms are built for d in {1, 2}", d);
  if (n < 1) return set_error(FK_EINVAL, "n = %lld < 1", (long long)n);
  if (!(eps >= 1e-14 && eps <= 1e-1)) return set_error(FK_EINVAL, "eps = %g outside [1e-14, 1e-1]", eps);
  if (precision != FK_FP64 && precision != FK_MIXED) return set_error(FK_EINVAL, "unknown precision %d", precision);
  if (kmax < 0 || n_ch < 1 || !x || !c || !out) return set_error(FK_EINVAL, "bad type-1 arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FK_TRY(capture_check(st, false, false, "fk_type1_noalloc"));
  EsPlan p;
  FK_TRY(make_es_plan(d, kmax, eps, 1.9, &p));
  const size_t G = (d == 1) ? static_cast<size_t>(p.N) : static_cast<size_t>(p.N) * p.N;
  const size_t K = 2 * static_cast<size_t>(kmax) + 1;
  const size_t elem = (precision == FK_FP64) ? sizeof(cplx<double>) : sizeof(cplx<float>);
  // layout: flags | corr | quadrature nodes | twiddles | grid | row-transform intermediate
  const size_t o_corr = 256;
  const size_t o_gl = align256(o_corr + sizeof(double) * K);
  const size_t o_tw = align256(o_gl + sizeof(double) * 2 * es_gl_nodes());
  const size_t o_grid = align256(o_tw + sizeof(double) * 2 * p.N);
  const size_t o_h = align256(o_grid + sizeof(double) * G * n_ch);
  const size_t need = align256(o_h + ((d == 2) ? elem * n_ch * p.N * K : 0));
  if (need > FK_NOALLOC_SCRATCH_BYTES)
    return set_error(FK_EINVAL,
                     "fk_type1_noalloc needs %zu bytes of scratch for d=%d kmax=%d n_ch=%d eps=%g (fine grid %d); "
                     "the built-in limit is %zu bytes",
                     need, d, kmax, n_ch, eps, p.N, static_cast<size_t>(FK_NOALLOC_SCRATCH_BYTES));
  void* base = nullptr;
  FK_TRY(scratch_address(&base));
  unsigned char* s = static_cast<unsigned char*>(base);
  unsigned* flags = reinterpret_cast<unsigned*>(s);
  double* corr = reinterpret_cast<double*>(s + o_corr);
  double* gl = reinterpret_cast<double*>(s + o_gl);
  double* tw = reinterpret_cast<double*>(s + o_tw);
  double* grid = reinterpret_cast<double*>(s + o_grid);
  FK_CUDA(cudaMemsetAsync(flags, 0, sizeof(unsigned), st));
  FK_TRY(es_correction_into(p, corr, gl, st));
  if (precision == FK_FP64) {
    FK_TRY(spread_atomic<double>(p, n, static_cast<const double*>(x), static_cast<const double*>(c), n_ch, false, grid,
                                 flags, st));
    FK_TRY(grid_to_modes_into<double>(p, grid, 0, n_ch, kmax, corr, 1.0, out, st, tw,
                                      reinterpret_cast<cplx<double>*>(s + o_h)));
  } else {
    FK_TRY(spread_atomic<float>(p, n, static_cast<const float*>(x), static_cast<const float*>(c), n_ch, false, grid,
                                flags, st));
    FK_TRY(grid_to_modes_into<float>(p, grid, 0, n_ch, kmax, corr, 1.0, out, st, tw,
                                     reinterpret_cast<cplx<float>*>(s + o_h)));
  }
  unsigned h = 0;
  FK_CUDA(cudaMemcpyAsync(&h, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  FK_CUDA(cudaStreamSynchronize(st));
  if (h & FLAG_RANGE) return set_error(FK_ERANGE, "a point lies outside [-3 pi, 3 pi)");
  if (h) return set_error(FK_EINTERNAL, "device flag 0x%x", h);
  return FK_OK;
}
