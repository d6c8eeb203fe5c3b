"""Host check of the stage kernel's shared-memory map (no GPU needed): for every tile shape
the library builds and every ragged extent of a tile, the cells the kernel fills (owned cells
and the cross-shaped halo) land on distinct in-range locations, and every cell a WENO window
or a face reads is one that was filled, at the location it was filled; and every vector
access of the grouped field layout is aligned to its size, for every instantiated field count
and tile. In 3-D the map stores
only the stencil cross (x-lines with both x halos, then the y and the z halos), so an error
there would silently mix two cells; in the x-z plane it is the plain box."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

DRIVER = r"""
#include <cstdio>
#include <map>
#include <set>
#include <tuple>
#include "paper_1901_02955_gb300/csrc/snap_stage.cuh"
using namespace snap;

template <class T, bool D3>
int check(int ex, int ey, int ez) {
  using B = Box<T, D3>;
  const int HY = D3 ? 3 : 0;
  std::map<int, std::tuple<int, int, int>> owner;
  std::set<std::tuple<int, int, int>> filled;
  int bad = 0;
  auto fill = [&](int bx, int by, int bz) {
    const int i = B::idx(bx, by, bz);
    const auto key = std::make_tuple(bx, by, bz);
    if (i < 0 || i >= B::NSTORE) { ++bad; return; }
    auto it = owner.find(i);
    if (it != owner.end() && it->second != key) ++bad;
    owner[i] = key;
    filled.insert(key);
  };
  auto read = [&](int bx, int by, int bz) {
    const int i = B::idx(bx, by, bz);
    const auto key = std::make_tuple(bx, by, bz);
    if (i < 0 || i >= B::NSTORE || !filled.count(key)) { ++bad; return; }
    if (owner[i] != key) ++bad;
  };
  for (int lz = 0; lz < ez; ++lz)
    for (int ly = 0; ly < ey; ++ly)
      for (int lx = 0; lx < ex; ++lx) fill(lx + 3, ly + HY, lz + 3);
  for (int r = 0; r < 6; ++r) {
    for (int lz = 0; lz < ez; ++lz)
      for (int ly = 0; ly < ey; ++ly) fill(r < 3 ? r : ex + r, ly + HY, lz + 3);
    if (D3)
      for (int lz = 0; lz < ez; ++lz)
        for (int lx = 0; lx < ex; ++lx) fill(lx + 3, r < 3 ? r : ey + r, lz + 3);
    for (int ly = 0; ly < ey; ++ly)
      for (int lx = 0; lx < ex; ++lx) fill(lx + 3, ly + HY, r < 3 ? r : ez + r);
  }
  const int e[3] = {ex, ey, ez};
  for (int d = 0; d < 3; ++d) {
    if (d == 1 && !D3) continue;
    const int fx = d == 0, fy = d == 1, fz = d == 2;
    for (int lz = -fz; lz < ez + fz; ++lz)
      for (int ly = -fy; ly < ey + fy; ++ly)
        for (int lx = -fx; lx < ex + fx; ++lx) {
          const int ld = fx ? lx : (fy ? ly : lz);
          if (ld > e[d]) continue;
          for (int k = -2; k <= 2; ++k) {
            read(lx + 3 + fx * k, ly + HY + fy * k, lz + 3 + fz * k);
            // the kernel maps 3-D y and z windows with the one-test forms
            if (D3 && fy && B::idx_y(lx + 3, ly + HY + k, lz + 3) != B::idx(lx + 3, ly + HY + k, lz + 3)) ++bad;
            if (D3 && fz && B::idx_z(lx + 3, ly + HY, lz + 3 + k) != B::idx(lx + 3, ly + HY, lz + 3 + k)) ++bad;
          }
        }
    for (int iz = 0; iz < ez + fz; ++iz)
      for (int iy = 0; iy < ey + fy; ++iy)
        for (int ix = 0; ix < ex + fx; ++ix) {
          read(ix + 3, iy + HY, iz + 3);
          read(ix + 3 - fx, iy + HY - fy, iz + 3 - fz);
        }
  }
  return bad;
}

template <class T, bool D3>
int all_extents() {
  int bad = 0;
  for (int ez = 1; ez <= T::TZ; ++ez)
    for (int ey = 1; ey <= T::TY; ++ey)
      for (int ex = 1; ex <= T::TX; ++ex) bad += check<T, D3>(ex, ey, ez);
  return bad;
}

// Every vector access of the grouped field layout (16-byte groups, then an 8-byte pair)
// lands on a multiple of its size, for every array of the stage's shared memory, every field
// and every location: the arrays' byte offsets plus SV::at.
template <class R, int NV, class T, bool D3, bool VISC>
int aligned() {
  using L = Lay<0, 0, D3>;  // only NV matters below
  using B = Box<T, D3>;
  using V = SV<R, NV>;
  const size_t prim = (sizeof(R) * NV * B::NSTORE + 15) / 16 * 16;
  const size_t visc = VISC ? (sizeof(R) * 2 * B::NSTORE + 15) / 16 * 16 : 0;
  const size_t half = (sizeof(R) * NV * B::NF + 15) / 16 * 16;
  const size_t bases[3] = {0, prim + visc, prim + visc + half};
  const int N[3] = {B::NSTORE, B::NF, B::NF};
  int bad = 0;
  (void)sizeof(L);
  for (int a = 0; a < 3; ++a)
    for (int i = 0; i < N[a]; ++i)
      for (int v = 0; v < NV; ++v) {
        const size_t byte = bases[a] + sizeof(R) * V::at(v, i, N[a]);
        const size_t width = v < V::P2 ? 16 : (v < V::P1 ? 8 : sizeof(R));
        const int first = v < V::P2 ? v % V::W == 0 : (v < V::P1 ? v == V::P2 : 1);
        if (first && byte % width) ++bad;
      }
  return bad;
}

int main() {
  int bad = 0;
  // the layouts and tiles the library instantiates: dry x-z (4 fields), moist x-z (7), dry
  // 3-D (5), moist 3-D (11), in FP32 and FP64
  bad += aligned<float, 4, TileT<64, 1, 14>, false, true>();
  bad += aligned<float, 4, TileT<32, 1, 14>, false, true>();
  bad += aligned<float, 4, TileT<128, 1, 14>, false, true>();
  bad += aligned<float, 4, TileT<64, 1, 28>, false, true>();
  bad += aligned<double, 4, TileT<32, 1, 28>, false, true>();
  bad += aligned<double, 4, TileT<32, 1, 14>, false, true>();
  bad += aligned<float, 7, TileT<32, 1, 14>, false, false>();
  bad += aligned<float, 7, TileT<64, 1, 6>, false, false>();
  bad += aligned<float, 7, TileT<16, 1, 30>, false, false>();
  bad += aligned<double, 7, TileT<32, 1, 14>, false, false>();
  bad += aligned<float, 5, TileT<8, 8, 4>, true, true>();
  bad += aligned<float, 5, TileT<16, 8, 2>, true, true>();
  bad += aligned<double, 5, TileT<8, 8, 4>, true, true>();
  bad += aligned<float, 11, TileT<8, 8, 4>, true, false>();
  bad += aligned<float, 11, TileT<16, 8, 2>, true, false>();
  bad += aligned<double, 11, TileT<8, 8, 4>, true, false>();
  if (bad) printf("misaligned %d\n", bad);
  bad += all_extents<TileT<8, 8, 4>, true>();
  bad += all_extents<TileT<16, 8, 2>, true>();
  bad += all_extents<TileT<32, 1, 14>, false>();
  bad += all_extents<TileT<64, 1, 14>, false>();
  bad += all_extents<TileT<32, 1, 28>, false>();
  bad += all_extents<TileT<16, 1, 30>, false>();
  bad += all_extents<TileT<64, 1, 6>, false>();
  printf("bad %d\n", bad);
  return bad != 0;
}
"""


def test_shared_memory_map_is_injective_and_covers_every_read(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("no nvcc")
    src = tmp_path / "map_check.cu"
    src.write_text(DRIVER)
    exe = tmp_path / "map_check"
    subprocess.check_call([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-gencode",
                           "arch=compute_103a,code=sm_103a", "-I", ROOT, str(src), "-o", str(exe)],
                          cwd=ROOT)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip() == "bad 0"
