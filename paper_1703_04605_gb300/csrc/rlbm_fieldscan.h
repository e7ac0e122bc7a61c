// Host-side validation of initial fields (rlbm_init, rlbm3_init): one pass
// over the caller's arrays that finds the first site violating n > 0, T > 0,
// |u| < 1 (all finite) and sums the density.  Large lattices are split into a
// fixed number of chunks scanned by worker threads; the partial sums are added
// in chunk order, so the mean is the same whatever the thread count.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <thread>
#include <vector>

namespace rlbm {

struct FieldScan {
  size_t first_bad;   // index of the first invalid site, or N if none
  double nsum;        // sum of n over all sites (meaningful when first_bad == N)
};

// uz may be NULL (2D lattices).
inline FieldScan scan_fields(const double* n, const double* ux, const double* uy, const double* uz,
                             const double* T, size_t N) {
  constexpr size_t kChunks = 64;
  constexpr size_t kSerialBelow = size_t(1) << 20;
  const size_t nchunk = N < kSerialBelow ? 1 : kChunks;
  const size_t len = (N + nchunk - 1) / nchunk;
  std::vector<size_t> bad(nchunk, N);
  std::vector<double> sum(nchunk, 0.0);
  auto scan = [&](size_t c) {
    const size_t lo = std::min(N, c * len), hi = std::min(N, lo + len);
    double s = 0.0;
    for (size_t i = lo; i < hi; ++i) {
      double v2 = ux[i] * ux[i] + uy[i] * uy[i];
      if (uz) v2 += uz[i] * uz[i];
      if (!(n[i] > 0) || !(T[i] > 0) || !(v2 < 1) || !std::isfinite(n[i]) || !std::isfinite(T[i])) {
        bad[c] = i;
        return;
      }
      s += n[i];
    }
    sum[c] = s;
  };
  if (nchunk == 1) {
    scan(0);
  } else {
    const unsigned hw = std::thread::hardware_concurrency();
    const size_t nthr = std::max<size_t>(1, std::min<size_t>(hw ? hw : 1, 16));
    std::vector<std::thread> pool;
    for (size_t t = 0; t < nthr; ++t)
      pool.emplace_back([&, t] {
        for (size_t c = t; c < nchunk; c += nthr) scan(c);
      });
    for (auto& th : pool) th.join();
  }
  FieldScan r{N, 0.0};
  for (size_t c = 0; c < nchunk; ++c) {
    if (bad[c] < N) {
      r.first_bad = bad[c];
      return r;
    }
    r.nsum += sum[c];
  }
  return r;
}

}  // namespace rlbm
