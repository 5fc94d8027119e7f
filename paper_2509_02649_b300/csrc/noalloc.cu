// fk_type1_noalloc: the type-1 transform for callers that cannot allocate device
// memory.
//
// fk_type1 takes its scratch (the upsampled grid, twiddles, correction factors,
// the 2-D row-transform intermediate, an error flag) from cudaMallocAsync.  Some
// callers cannot allocate at call time: a process whose device memory is wholly
// reserved by its own pool allocator, or a service whose policy forbids device
// allocation after start-up.  This variant takes all of that scratch from one
// file-scope device array of FK_NOALLOC_SCRATCH_BYTES instead.  Every GPU on which
// the first call is made holds that array until the process exits.
//
// Set-up, once per device, in the first call on that device (with it current):
//  * the array's device address is looked up with cudaGetSymbolAddress (in host code
//    the array's name is only a host-side stand-in, not a device address).  With the
//    CUDA runtime's lazy module loading this lookup is also what loads the module and
//    places the array in device memory;
//  * the kernels later calls launch are loaded (cudaFuncGetAttributes), so that no
//    later call needs device memory for code;
//  * the Gauss-Legendre nodes of the correction factors are computed into the array.
// That first call therefore needs about FK_NOALLOC_SCRATCH_BYTES of free device memory
// plus the code: make it at start-up, before the caller reserves its memory and
// before any stream capture.
//
// All calls share the array and it keeps the last call's contents.  The grid and the
// flag word are cleared on every call; the quadrature nodes stay from the set-up, and
// the correction factors and twiddles of the last call's plan are reused when the
// next call has the same plan.  Calls whose work overlaps on the GPU (different
// streams, or host threads calling concurrently) race on the array.  The spreading
// step is the atomic form for both precisions.  The paper has no counterpart to this
// entry point.
#include "fk_internal.cuh"

#include <mutex>

namespace fk {
namespace {

constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[FK_NOALLOC_SCRATCH_BYTES];

// per device: the array's address, and the plan whose correction factors and twiddles
// the array holds (kmax < 0: none yet)
struct DevState {
  void* addr = nullptr;
  int kmax = -1, N = 0, w = 0;
  double beta = 0.0;
};
std::mutex g_mutex;
DevState g_dev[MAX_DEVICES];

size_t align256(size_t v) { return (v + 255) & ~static_cast<size_t>(255); }

// layout: flags | quadrature nodes | corr | twiddles | grid | row-transform intermediate
constexpr size_t O_GL = 256;
size_t o_corr() { return align256(O_GL + sizeof(double) * 2 * es_gl_nodes()); }

fk_status setup_device(int dev, cudaStream_t st, DevState* ds) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    return set_error(FK_ECUDA,
                     "set-up of fk_type1_noalloc on device %d failed: cudaGetSymbolAddress: %s.  The first call "
                     "on a device loads the library's code and places its %zu-byte scratch array; make it at "
                     "start-up, before device memory is reserved elsewhere",
                     dev, cudaGetErrorString(e), static_cast<size_t>(FK_NOALLOC_SCRATCH_BYTES));
  }
  fk_status rc = preload_es_kernels();
  if (rc == FK_OK) rc = preload_spread_atomic_kernels();
  if (rc == FK_OK) rc = preload_modes_kernels();
  if (rc != FK_OK)
    return set_error(rc, "set-up of fk_type1_noalloc on device %d: loading its kernels failed (%s); make the "
                         "first call at start-up, before device memory is reserved elsewhere",
                     dev, fk_last_error());
  unsigned char* s = static_cast<unsigned char*>(p);
  FK_TRY(es_gl_nodes_into(reinterpret_cast<double*>(s + O_GL), st));
  ds->addr = p;
  ds->kmax = -1;
  return FK_OK;
}

}  // namespace
}  // namespace fk

using namespace fk;

extern "C" fk_status fk_type1_noalloc(int d, int64_t n, const void* x, const void* c, int n_ch, int kmax, double eps,
                                      int precision, double* out, void* stream) {
  clear_error();
  // the checks of fk_type1, plus the dimensions this entry point is built for
  FK_TRY(check_common(d, n, 0, eps, precision));
  if (d > 2) return set_error(FK_EINVAL, "d = %d: fk_type1_noalloc is built for d in {1, 2}", d);
  if (kmax < 0 || n_ch < 1 || !x || !c || !out) return set_error(FK_EINVAL, "bad type-1 arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FK_TRY(capture_check(st, false, false, "fk_type1_noalloc"));
  EsPlan p;
  FK_TRY(make_es_plan(d, kmax, eps, 1.9, &p));
  const size_t G = (d == 1) ? static_cast<size_t>(p.N) : static_cast<size_t>(p.N) * p.N;
  const size_t K = 2 * static_cast<size_t>(kmax) + 1;
  const size_t elem = (precision == FK_FP64) ? sizeof(cplx<double>) : sizeof(cplx<float>);
  const size_t oc = o_corr();
  const size_t o_tw = align256(oc + sizeof(double) * K);
  const size_t o_grid = align256(o_tw + sizeof(double) * 2 * p.N);
  const size_t o_h = align256(o_grid + sizeof(double) * G * n_ch);
  const size_t need = align256(o_h + ((d == 2) ? elem * n_ch * p.N * K : 0));
  if (need > FK_NOALLOC_SCRATCH_BYTES)
    return set_error(FK_EINVAL,
                     "fk_type1_noalloc needs %zu bytes of scratch for d=%d kmax=%d n_ch=%d eps=%g (fine grid %d); "
                     "the built-in limit is %zu bytes",
                     need, d, kmax, n_ch, eps, p.N, static_cast<size_t>(FK_NOALLOC_SCRATCH_BYTES));
  int dev = 0;
  FK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES) return set_error(FK_EINVAL, "device %d beyond the supported %d", dev, MAX_DEVICES);
  std::lock_guard<std::mutex> lock(g_mutex);
  DevState& ds = g_dev[dev];
  if (!ds.addr) FK_TRY(setup_device(dev, st, &ds));
  unsigned char* s = static_cast<unsigned char*>(ds.addr);
  unsigned* flags = reinterpret_cast<unsigned*>(s);
  const double* gl = reinterpret_cast<const double*>(s + O_GL);
  double* corr = reinterpret_cast<double*>(s + oc);
  double* tw = reinterpret_cast<double*>(s + o_tw);
  double* grid = reinterpret_cast<double*>(s + o_grid);
  FK_CUDA(cudaMemsetAsync(flags, 0, sizeof(unsigned), st));
  // correction factors and twiddles: kept from the last call when its plan was the same
  // (they sit in front of every grid, so no call's grid overwrote them since)
  const bool same_plan = ds.kmax == p.kmax && ds.N == p.N && ds.w == p.w && ds.beta == p.beta;
  if (!same_plan) {
    ds.kmax = -1;
    FK_TRY(es_correction_from_nodes(p, corr, gl, st));
    FK_TRY(fft_twiddles(p.N, tw, st));
    ds.kmax = p.kmax;
    ds.N = p.N;
    ds.w = p.w;
    ds.beta = p.beta;
  }
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
