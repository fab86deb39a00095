// Run-time compiled grid potentials: CUDA C source from the caller, compiled with NVRTC
// for this GPU, evaluated once at every grid point and installed as a static grid
// potential (the user potential() of Sec. 3.2.3 of arXiv:1306.3247, which the paper links
// into its program at build time). NVRTC is opened with dlopen when first needed, so the
// library loads on machines without it.
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "wp_internal.h"

namespace {

struct Nvrtc {
  bool ok = false;
  std::string why;
  nvrtcResult (*create)(nvrtcProgram*, const char*, const char*, int, const char* const*, const char* const*);
  nvrtcResult (*compile)(nvrtcProgram, int, const char* const*);
  nvrtcResult (*log_size)(nvrtcProgram, size_t*);
  nvrtcResult (*log)(nvrtcProgram, char*);
  nvrtcResult (*cubin_size)(nvrtcProgram, size_t*);
  nvrtcResult (*cubin)(nvrtcProgram, char*);
  nvrtcResult (*destroy)(nvrtcProgram*);
};

const Nvrtc& nvrtc() {
  static Nvrtc n;
  static std::once_flag once;
  std::call_once(once, [] {
    const char* names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13"};
    void* lib = nullptr;
    for (const char* nm : names)
      if ((lib = dlopen(nm, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
    if (!lib) {
      n.why = "NVRTC library not found";
      return;
    }
    bool all = true;
    auto get = [&](auto& fp, const char* sym) {
      fp = reinterpret_cast<std::remove_reference_t<decltype(fp)>>(dlsym(lib, sym));
      all = all && fp != nullptr;
    };
    get(n.create, "nvrtcCreateProgram");
    get(n.compile, "nvrtcCompileProgram");
    get(n.log_size, "nvrtcGetProgramLogSize");
    get(n.log, "nvrtcGetProgramLog");
    get(n.cubin_size, "nvrtcGetCUBINSize");
    get(n.cubin, "nvrtcGetCUBIN");
    get(n.destroy, "nvrtcDestroyProgram");
    n.ok = all;
    if (!all) n.why = "NVRTC entry points missing";
  });
  return n;
}

// The grid kernel appended to the caller's source: point i of the row-major grid (last
// axis fastest) at coordinates xmin_d + i_d dx_d.
const char* kGridKernel = R"(
extern "C" __global__ void wp_user_grid(double* V, long long n, int ndim, int l1, int l2,
                                        double a0, double a1, double a2, double d0, double d1, double d2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    long long r = i;
    long long i2 = 0, i1 = 0;
    if (ndim > 2) { i2 = r & ((1LL << l2) - 1); r >>= l2; }
    if (ndim > 1) { i1 = r & ((1LL << l1) - 1); r >>= l1; }
    const double x = a0 + (double)r * d0;
    const double y = ndim > 1 ? a1 + (double)i1 * d1 : 0.0;
    const double z = ndim > 2 ? a2 + (double)i2 * d2 : 0.0;
    V[i] = wp_user_potential(x, y, z);
  }
}
)";

int ilog2i(int64_t v) {
  int l = 0;
  while ((int64_t(1) << l) < v) l++;
  return l;
}

}  // namespace

extern "C" wp_status wp_set_potential_source(wp_handle* h, const char* src) {
  if (!h || !src) return wp::handle_set_error(h, WP_EINVAL, "NULL argument");
  const Nvrtc& nv = nvrtc();
  if (!nv.ok) return wp::handle_set_error(h, WP_EUNSUPPORTED, nv.why.c_str());
  int ndim = 0;
  int64_t n[3];
  double xmin[3], dx[3];
  void* stream = nullptr;
  wp::handle_geometry(h, &ndim, n, xmin, dx, &stream);
  int dev = 0, major = 0, minor = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  // architecture-specific target (sm_103a on GB300)
  const std::string arch = "--gpu-architecture=sm_" + std::to_string(major * 10 + minor) + "a";
  const std::string code = std::string(src) + kGridKernel;
  nvrtcProgram prog = nullptr;
  if (nv.create(&prog, code.c_str(), "wp_user_potential.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS)
    return wp::handle_set_error(h, WP_ENOMEM, "NVRTC: cannot create the program");
  const char* opts[] = {arch.c_str(), "--std=c++17"};
  const nvrtcResult cr = nv.compile(prog, 2, opts);
  if (cr != NVRTC_SUCCESS) {
    size_t ls = 0;
    nv.log_size(prog, &ls);
    std::string log(ls, '\0');
    if (ls) nv.log(prog, &log[0]);
    nv.destroy(&prog);
    return wp::handle_set_error(h, WP_EINVAL, ("potential source does not compile: " + log).c_str());
  }
  size_t nb = 0;
  nv.cubin_size(prog, &nb);
  std::vector<char> cubin(nb);
  nv.cubin(prog, cubin.data());
  nv.destroy(&prog);

  cudaLibrary_t lib = nullptr;
  cudaKernel_t kern = nullptr;
  cudaError_t e = cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
  if (e == cudaSuccess) e = cudaLibraryGetKernel(&kern, lib, "wp_user_grid");
  if (e != cudaSuccess) {
    if (lib) cudaLibraryUnload(lib);
    return wp::handle_set_error(h, WP_ECUDA, cudaGetErrorString(e));
  }
  const int64_t N = n[0] * n[1] * n[2];
  double* V = nullptr;
  e = cudaMalloc(&V, (size_t)N * sizeof(double));
  if (e != cudaSuccess) {
    cudaLibraryUnload(lib);
    return wp::handle_set_error(h, WP_ENOMEM, "grid allocation");
  }
  long long nn = N;
  int nd = ndim, l1 = ilog2i(n[1]), l2 = ilog2i(n[2]);
  double a0 = xmin[0], a1 = xmin[1], a2 = xmin[2], d0 = dx[0], d1 = dx[1], d2 = dx[2];
  void* args[] = {&V, &nn, &nd, &l1, &l2, &a0, &a1, &a2, &d0, &d1, &d2};
  int64_t blocks = (N + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  e = cudaLaunchKernel((const void*)kern, dim3((unsigned)blocks), dim3(256), args, 0, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  wp_status st = WP_OK;
  if (e != cudaSuccess)
    st = wp::handle_set_error(h, WP_ECUDA, cudaGetErrorString(e));
  else
    st = wp_set_potential_grid(h, V, 1);
  cudaStreamSynchronize((cudaStream_t)stream);
  cudaFree(V);
  cudaLibraryUnload(lib);
  return st;
}
