// Host-side harness around the library's peak search (split_walk,
// split_recursive and keep_piece in pv_device.cuh), so CPU tests can compare it with the oracle on
// many histograms.  Test code only: proto-clusters are found with a plain loop
// and every proto-cluster is walked (no early skip).
#include <cstdint>
#include <vector>

#include "pv_device.cuh"

extern "C" int harness_seeds(const uint32_t* N, int nbins, uint32_t thr, uint32_t t_pp,
                             uint32_t t_gas, int dip_num, int dip_den, int gas_bin,
                             int split_mode, int* lo, int* hi, int* bin, int cap) {
  pvdev::Consts C{};
  C.nbins = nbins;
  C.thr = thr;
  C.t_pp = t_pp;
  C.t_gas = t_gas;
  C.dip_num = dip_num;
  C.dip_den = dip_den;
  C.gas_bin = gas_bin;
  int n = 0;
  std::vector<int16_t> mark(nbins);   // the recursive split's per-bin scratch
  for (int i = 0; i < nbins; ++i) {
    if (!(N[i] > thr)) continue;
    const int a = i;
    while (i + 1 < nbins && N[i + 1] > thr) ++i;
    const int b = i;
    uint64_t total = 0;
    for (int j = a; j <= b; ++j) total += N[j];
    auto emit = [&](int l, int h, uint64_t integral, int im) {
      if (pvdev::keep_piece(integral, im, C)) {
        if (n < cap) {
          lo[n] = l;
          hi[n] = h;
          bin[n] = im;
        }
        ++n;
      }
    };
    if (split_mode == PV_SPLIT_RECURSIVE)
      pvdev::split_pieces<PV_SPLIT_RECURSIVE>(N, a, b, total, C, emit, mark.data());
    else
      pvdev::split_pieces<PV_SPLIT_ZORDER>(N, a, b, total, C, emit, mark.data());
  }
  return n;
}
