"""The batched single-pass CG kernel's plan, checked on the CPU.

The batched kernel runs the float32 correction solves of many systems in one
launch.  Its host plan (exported by libparo.so) gives the candidate geometries
of a batch (``paro::cg2b_candidates``: tile, nodes a thread, orbital block width,
ring depth, shared memory) and, for each, the work tables
(``paro::cg2b_tables``): the orbital blocks of every system and their items,
tile columns cut into z-chunks.  A host program linked against the library
prints them for batches shaped like the uneven-systems workload (meshes 32^3 to
96^3, 4 to 48 orbitals) and for ragged small meshes, and this test checks what
the kernel relies on: every interior node of every orbital block in exactly one
item, chunks inside the interior planes, blocks that cover each system's
orbitals with 1 to G4 groups, TMA boxes of at most 256 elements with inner
extents and start coordinates on 16-byte multiples, slot transaction counts
below 2^20, thread and shared-memory limits of one CTA per SM, and enough items
for every CTA.  Needs nvcc and the built library, no GPU.
"""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1405_0260_gb300", "csrc")
LIBDIR = os.path.join(ROOT, "paper_1405_0260_gb300")

SRC = r'''
#include <cstdio>
#include <vector>
#include "cg.cuh"
using namespace paro;
static Grid grid_of(int nx, int ny, int nz) {
  Grid g{};
  g.nx = nx; g.ny = ny; g.nz = nz;
  g.Px = nx + 1; g.Py = ny + 1; g.Pz = nz + 1;
  g.G = (long long)g.Px * g.Py * g.Pz;
  g.nI = (nx - 1) * (ny - 1) * (nz - 1);
  return g;
}
int main() {
  // batches: (nx, ny, nz, N) per system
  const std::vector<std::vector<std::array<int, 4>>> batches = {
      {{32, 32, 32, 4}, {48, 48, 48, 13}, {64, 64, 64, 20}, {96, 96, 96, 46}, {32, 32, 32, 48}, {48, 48, 48, 7}},
      {{13, 13, 13, 10}, {11, 11, 11, 5}, {17, 17, 17, 20}, {9, 9, 9, 4}},
      {{5, 7, 6, 4}, {33, 17, 65, 12}, {10, 12, 9, 9}},
      {{64, 64, 64, 20}, {64, 64, 64, 20}}};
  int b = 0;
  for (const auto& bt : batches) {
    CG2BPlan P;
    for (const auto& s : bt) {
      CG2BSysDesc d{};
      d.g = grid_of(s[0], s[1], s[2]);
      d.N = s[3];
      d.Np = (s[3] + 3) / 4 * 4;
      d.dpitch = d.g.Px + 8;
      P.desc.push_back(d);
    }
    std::vector<K1Geom> cand;
    cg2b_candidates(&P, &cand);
    std::printf("B %d %zu\n", b, cand.size());
    for (size_t c = 0; c < cand.size(); ++c) {
      K1Geom G = cand[c];
      G.grid = 152;
      std::vector<CG2BJob> jobs;
      std::vector<int4> items;
      int zlen = 0;
      cg2b_tables(P.desc, G, &jobs, &items, &zlen);
      // coverage: interior nodes of each job summed over its items, bounds
      long long bad = 0, covered_ok = 1, orb_ok = 1;
      std::vector<long long> cover(jobs.size(), 0);
      for (size_t i = 0; i < items.size(); ++i) {
        const int4 it = items[i];
        const CG2BJob& J = jobs[it.x];
        const Grid& g = P.desc[J.sys].g;
        const int x0 = 1 + it.y * G.TX, y0 = 1 + it.z * G.TY, z0 = 1 + it.w * zlen;
        int z1 = z0 + zlen;
        if (z1 > g.nz) z1 = g.nz;
        const int x1 = x0 + G.TX < g.nx ? x0 + G.TX : g.nx, y1 = y0 + G.TY < g.ny ? y0 + G.TY : g.ny;
        if (x0 > g.nx - 1 || y0 > g.ny - 1 || z0 > g.nz - 1 || z0 >= z1 || (int)i < J.it0 || (int)i >= J.it0 + J.nit)
          ++bad;
        if (((x0 - 1) * 4 * 4) % 16 || ((x0 - 1) * 4) % 16) ++bad;  // vector and D^-1 box starts (bytes)
        cover[it.x] += (long long)(x1 - x0) * (y1 - y0) * (z1 - z0);
      }
      for (size_t j = 0; j < jobs.size(); ++j)
        if (cover[j] != P.desc[jobs[j].sys].g.nI) covered_ok = 0;
      for (size_t s = 0; s < P.desc.size(); ++s) {
        int groups = 0, prev_ob = -1;
        for (const auto& J : jobs)
          if (J.sys == (int)s) {
            if (J.ng < 1 || J.ng > G.G4 || J.ob != prev_ob + 1) orb_ok = 0;
            prev_ob = J.ob;
            groups += J.ng;
          }
        if (4 * groups != P.desc[s].Np) orb_ok = 0;
      }
      std::printf("G %d %zu %d %d %d %d %d %d %zu %d %d %d %d %d %u %d %zu %zu %lld %lld %lld\n", b, c, G.TX, G.TY,
                  G.npt, G.G4, G.nthr, G.slots, G.smem, G.DX, G.off_p, G.off_s, G.off_d, G.off_w, (unsigned)G.tx_bytes,
                  zlen, items.size(), jobs.size(), bad, covered_ok, orb_ok);
    }
    ++b;
  }
  return 0;
}
'''


@pytest.fixture(scope="module")
def plans():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    lib = os.path.join(LIBDIR, "libparo.so")
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    if not os.path.exists(lib):
        import __graft_entry__

        __graft_entry__.build()
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "plan2b.cu"), os.path.join(d, "plan2b")
        with open(src, "w") as f:
            f.write(SRC.replace("#include <vector>", "#include <array>\n#include <vector>"))
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-I", CSRC,
                        "-I", os.path.join(ROOT, "include"), src, "-o", exe, "-L", LIBDIR, "-lparo",
                        "-Xlinker", "-rpath=" + LIBDIR, "-lcuda"], check=True, capture_output=True, timeout=600)
        out = subprocess.run([exe], capture_output=True, text=True, check=True, timeout=600).stdout
    counts, geoms = {}, []
    for line in out.splitlines():
        t = line.split()
        if t[0] == "B":
            counts[int(t[1])] = int(t[2])
        elif t[0] == "G":
            v = [int(x) for x in t[1:]]
            keys = ("batch cand TX TY npt G4 nthr slots smem DX off_p off_s off_d off_w tx_bytes zlen nitems njobs "
                    "bad covered orbitals").split()
            geoms.append(dict(zip(keys, v)))
    return counts, geoms


def test_every_batch_has_candidates(plans):
    counts, geoms = plans
    assert set(counts) == {0, 1, 2, 3}
    assert all(c >= 4 for c in counts.values()), counts
    assert len(geoms) == sum(counts.values())


def test_items_cover_every_node_of_every_orbital_block_once(plans):
    _, geoms = plans
    for g in geoms:
        assert g["bad"] == 0, g
        assert g["covered"] == 1, g
        assert g["orbitals"] == 1, g


def test_tma_boxes_and_slots_obey_the_hardware_rules(plans):
    _, geoms = plans
    for g in geoms:
        TX, TY = g["TX"], g["TY"]
        # vector box (4 (TX+2) floats, TY+2 rows), D^-1 box (DX floats), weights box (28, TX, TY)
        for extent in (4 * (TX + 2), TY + 2, g["DX"], 28, TX, TY):
            assert extent <= 256, g
        assert (4 * (TX + 2) * 4) % 16 == 0 and (g["DX"] * 4) % 16 == 0 and (28 * 4) % 16 == 0, g
        assert TX % 4 == 0, g  # D^-1 box starts at x0 - 1 = tile index x TX floats
        for off in (g["off_p"], g["off_s"], g["off_d"], g["off_w"]):
            assert off % 128 == 0, g
        assert g["tx_bytes"] < 1 << 20, g
        assert 3 <= g["slots"] <= 6, g


def test_launch_shape_fits_one_cta_per_sm(plans):
    _, geoms = plans
    for g in geoms:
        threads = g["nthr"] * g["G4"] + 32
        assert threads <= (384 if g["npt"] == 2 else 512), g
        assert g["nthr"] % 32 == 0, g  # a warp holds one group slot (per-warp partial sums)
        assert g["smem"] <= 227 * 1024 - 1024, g
        assert 1 <= g["G4"] <= 8, g


def test_enough_items_for_every_cta(plans):
    _, geoms = plans
    for g in geoms:
        # whole columns, or chunks halved down to no fewer than 9 planes (2 halo planes each)
        assert g["zlen"] >= 8, g
    # the uneven-systems batch has plenty of items at its untuned default
    first = [g for g in geoms if g["batch"] == 0][0]
    assert first["nitems"] >= 8 * 152, first
