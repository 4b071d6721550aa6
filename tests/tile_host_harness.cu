// Host harness for the step kernel's tile geometry: the cell and face counts of every tile shape and
// the ring cells its ring phase evaluates, read on the CPU from the same templates the kernel uses.
#include "gks_step.cuh"

namespace {

constexpr int kInfo = 13;

template <int D, int V> int info(int* o) {
  using G = gks::TileGeom<D, V>;
  const int v[kInfo] = {G::X,   G::Y,   G::Z,   G::T,   G::RX, G::RY, G::RZ,
                        G::NR,  G::NFX, G::NFY, G::NFZ, G::NF, gks::ring_used<D, G>()};
  for (int i = 0; i < kInfo; ++i) o[i] = v[i];
  return kInfo;
}

template <int D, int V> int slots(int* o) {
  using G = gks::TileGeom<D, V>;
  constexpr int n = gks::ring_used<D, G>();
  for (int s = 0; s < n; ++s) o[s] = gks::ring_slot<D, G>(s);
  return n;
}

}  // namespace

#define GKS_TILE_CASES(fn, out)  \
  switch (D * 16 + V) {          \
    case 16 + 0: return fn<1, 0>(out); \
    case 16 + 1: return fn<1, 1>(out); \
    case 16 + 2: return fn<1, 2>(out); \
    case 32 + 0: return fn<2, 0>(out); \
    case 32 + 1: return fn<2, 1>(out); \
    case 32 + 2: return fn<2, 2>(out); \
    case 32 + 3: return fn<2, 3>(out); \
    case 32 + 4: return fn<2, 4>(out); \
    case 32 + 5: return fn<2, 5>(out); \
    case 32 + 6: return fn<2, 6>(out); \
    case 32 + 7: return fn<2, 7>(out); \
    case 32 + 8: return fn<2, 8>(out); \
    case 48 + 0: return fn<3, 0>(out); \
    case 48 + 1: return fn<3, 1>(out); \
    case 48 + 2: return fn<3, 2>(out); \
    case 48 + 3: return fn<3, 3>(out); \
    default: return -1;          \
  }

// Geometry of tile variant V in D dimensions: X, Y, Z, threads, ring box RX, RY, RZ, ring cells,
// faces along x, y, z, all faces, ring cells evaluated; returns the count written or -1.
extern "C" int tile_info(int D, int V, int* out) { GKS_TILE_CASES(info, out) }

// Ring-box indices (ri + RX (rj + RY rk)) of the ring cells the ring phase evaluates, in its order;
// returns their number or -1.
extern "C" int tile_ring_slots(int D, int V, int* out) { GKS_TILE_CASES(slots, out) }
