// Host-side harness around the library's peak search (split_walk,
// split_recursive, split_recursive_descend and keep_piece in pv_device.cuh), so CPU tests
// can compare it with the oracle on many histograms (the recursive split both with its
// scratch and without).  Test code only: proto-clusters are found with a plain loop
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
  std::vector<int16_t> mark(nbins);   // the recursive split's scratch (relative to a run)
  struct Piece {
    int l, h, im;
    uint64_t integral;
    bool operator==(const Piece& o) const {
      return l == o.l && h == o.h && im == o.im && integral == o.integral;
    }
  };
  bool same = true;
  for (int i = 0; i < nbins; ++i) {
    if (!(N[i] > thr)) continue;
    const int a = i;
    while (i + 1 < nbins && N[i + 1] > thr) ++i;
    const int b = i;
    uint64_t total = 0;
    for (int j = a; j <= b; ++j) total += N[j];
    // the recursive split with its scratch and without (descending for every
    // piece): the same pieces
    std::vector<Piece> pm, pd;
    auto emit_m = [&](int l, int h, uint64_t integral, int im) { pm.push_back({l, h, im, integral}); };
    auto emit_d = [&](int l, int h, uint64_t integral, int im) { pd.push_back({l, h, im, integral}); };
    if (split_mode == PV_SPLIT_RECURSIVE) {
      pvdev::split_pieces<PV_SPLIT_RECURSIVE>(N, a, b, total, C, emit_m, mark.data());
      pvdev::split_pieces<PV_SPLIT_RECURSIVE>(N, a, b, total, C, emit_d, nullptr);
      if (!(pm == pd)) same = false;
    } else {
      pvdev::split_pieces<PV_SPLIT_ZORDER>(N, a, b, total, C, emit_m, nullptr);
    }
    for (const Piece& q : pm) {
      if (pvdev::keep_piece(q.integral, q.im, C)) {
        if (n < cap) {
          lo[n] = q.l;
          hi[n] = q.h;
          bin[n] = q.im;
        }
        ++n;
      }
    }
  }
  if (!same) return -2;   // the recursive split with and without scratch disagree
  return n;
}
