// Host build of the FP64 fused multiply-add butterflies and their twiddle records
// (wp_fft_f64.h), driven through the same Stockham stage order and index map as the
// fixed-size device transform, for the CPU tests. Reads logn, direction and 2^logn
// complex doubles from stdin (binary); writes the unnormalised transform to stdout.
#define __host__
#define __device__
#define __forceinline__ inline
#include <cstdio>
#include <vector>

#include "wp_fft_f64.h"

using wp::cx;

int main() {
  int32_t hdr[2];
  if (fread(hdr, sizeof(hdr), 1, stdin) != 1) return 2;
  const int logn = hdr[0];
  const bool inv = hdr[1] != 0;
  if (logn < 1 || logn > 16) return 2;
  const int n = 1 << logn;
  std::vector<cx<double>> x(n), y(n);
  if (fread(x.data(), sizeof(cx<double>), n, stdin) != (size_t)n) return 2;
  std::vector<unsigned char> tab(2 * (size_t)wp::wp_fma_dir_bytes(logn) + 16);
  wp::wp_fma_build_tables(logn, tab.data());
  const unsigned char* dir = tab.data() + (inv ? wp::wp_fma_dir_bytes(logn) : 0);
  int ls = 0;
  while (ls < logn) {
    const int lr = wp::wp_stage_radix_log(logn, ls), R = 1 << lr, nr = n >> lr, ns = 1 << ls;
    for (int j = 0; j < nr; j++) {
      cx<double> v[8];
      for (int r = 0; r < R; r++) v[r] = x[j + r * nr];
      const int jm = j & (ns - 1);
      const unsigned char* rec = dir + wp::wp_fma_stage_offset(logn, ls) + (size_t)jm * wp::wp_fma_rec_bytes(lr);
      if (ls == 0) {
        if (R == 8) {
          inv ? wp::fma_dft8_first<true>(v) : wp::fma_dft8_first<false>(v);
        } else if (R == 4) {
          cx<double> d[4];
          inv ? wp::plain_dft4<true>(v[0], v[1], v[2], v[3], d) : wp::plain_dft4<false>(v[0], v[1], v[2], v[3], d);
          for (int r = 0; r < 4; r++) v[r] = d[r];
        } else {
          const cx<double> a = v[0];
          v[0] = wp::cxd(a.re + v[1].re, a.im + v[1].im);
          v[1] = wp::cxd(a.re - v[1].re, a.im - v[1].im);
        }
      } else if (R == 8) {
        const wp::Fma8* q = reinterpret_cast<const wp::Fma8*>(rec);
        inv ? wp::fma_dft8<true>(v, *q) : wp::fma_dft8<false>(v, *q);
      } else if (R == 4) {
        const wp::Fma4* q = reinterpret_cast<const wp::Fma4*>(rec);
        inv ? wp::fma_dft4<true>(v, *q) : wp::fma_dft4<false>(v, *q);
      } else {
        const wp::Fma2* q = reinterpret_cast<const wp::Fma2*>(rec);
        inv ? wp::fma_dft2<true>(v, *q) : wp::fma_dft2<false>(v, *q);
      }
      const int d0 = ((j >> ls) << (ls + lr)) + jm;
      for (int r = 0; r < R; r++) y[d0 + (r << ls)] = v[r];
    }
    x.swap(y);
    ls += lr;
  }
  fwrite(x.data(), sizeof(cx<double>), n, stdout);
  return 0;
}
