"""The tiled CG kernel's launch geometry, checked on the CPU.

The single-reduction CG kernel stages r, w and s (with a one-node halo), the
Jacobi diagonal and the packed operator weights of every input plane by TMA
into a ring of shared-memory slots, and splits the column-planes of the mesh
over a grid of CTAs.  Its plan is computed on the host by
``paro::cg1_candidates`` (exported by libparo.so).  This test compiles a small
host program against the library, asks for the candidate geometries of many
meshes (cubic, uneven, odd, small and the largest workload's 192^3) and
orbital counts (4 to 256), and checks every one against the limits the kernel
relies on: TMA boxes of at most 256 elements per dimension whose inner extent
and start coordinate are multiples of 16 bytes, 128-byte aligned slots, a
transaction count below the mbarrier's 2^20, at most 1024 threads and 227 KB of
shared memory per CTA, column tiles that cover the interior nodes, orbital
blocks that cover the orbitals, and a split that hands out every column-plane
exactly once in order.  The two-phase CG kernel (the float64 path) gets the
same checks from ``paro::cg_plan_geometry`` in float32 and float64.  The same
program prints the library's constant mass
stencil, which is compared with a row of the oracle's assembled mass matrix.
Needs nvcc and the built library, no GPU.
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
int main() {
  const int meshes[][3] = {{4, 4, 4}, {5, 7, 6}, {10, 12, 9}, {16, 16, 16}, {33, 17, 65}, {32, 48, 64},
                           {64, 64, 64}, {96, 96, 96}, {128, 128, 128}, {192, 192, 192}};
  for (auto& m : meshes) {
    Grid g{};
    g.nx = m[0]; g.ny = m[1]; g.nz = m[2];
    g.Px = g.nx + 1; g.Py = g.ny + 1; g.Pz = g.nz + 1;
    g.G = (long long)g.Px * g.Py * g.Pz;
    g.nI = (g.nx - 1) * (g.ny - 1) * (g.nz - 1);
    g.hx = g.hy = g.hz = 1.0;
    for (int Np = 4; Np <= 256; Np += 4) {
      std::vector<K1Geom> c;
      cg1_candidates(g, Np, 152, &c);
      std::printf("N %d %d %d %d %zu\n", g.nx, g.ny, g.nz, Np, c.size());
      for (const K1Geom& G : c) {
        long long F = (long long)G.nob * G.ncx * G.ncy * (g.nz - 1);
        int mono = 1;
        long long maxcost = 0;
        for (int k = 0; k < G.grid; ++k) {
          if (G.split[k + 1] < G.split[k]) mono = 0;
          long long a = G.split[k], b = G.split[k + 1], cost = 0;
          while (a < b) {  // planes plus two halo planes per column segment
            long long end = (a / (g.nz - 1) + 1) * (g.nz - 1);
            long long e = end < b ? end : b;
            cost += (e - a) + 2;
            a = e;
          }
          if (cost > maxcost) maxcost = cost;
        }
        std::printf("G %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %u %zu %d %lld %lld %d %lld\n",
                    g.nx, g.ny, g.nz, Np, G.TX, G.TY, G.DX, G.ncx, G.ncy, G.nob, G.grid, G.G4, G.npt, G.nthr,
                    G.off_p, G.off_s, G.off_d, G.off_w, G.slot_bytes, (unsigned)G.tx_bytes, G.smem, G.split[0],
                    (long long)G.split[G.grid], F, mono, maxcost);
      }
    }
  }
  // the single-pass CG kernel (group-major vectors): its candidates
  for (auto& m : meshes) {
    Grid g{};
    g.nx = m[0]; g.ny = m[1]; g.nz = m[2];
    g.Px = g.nx + 1; g.Py = g.ny + 1; g.Pz = g.nz + 1;
    g.G = (long long)g.Px * g.Py * g.Pz;
    g.nI = (g.nx - 1) * (g.ny - 1) * (g.nz - 1);
    for (int Np = 4; Np <= 256; Np += 4) {
      std::vector<K1Geom> c;
      cg2_candidates(g, Np, 152, &c);
      std::printf("n %d %d %d %d %zu\n", g.nx, g.ny, g.nz, Np, c.size());
      for (const K1Geom& G : c) {
        long long F = (long long)G.nob * G.ncx * G.ncy * (g.nz - 1);
        int mono = 1;
        for (int k = 0; k < G.grid; ++k)
          if (G.split[k + 1] < G.split[k]) mono = 0;
        std::printf("C %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %u %zu %d %lld %lld %d %d\n",
                    g.nx, g.ny, g.nz, Np, G.TX, G.TY, G.DX, G.ncx, G.ncy, G.nob, G.grid, G.G4, G.npt, G.nthr,
                    G.off_p, G.off_s, G.off_d, G.off_w, G.slot_bytes, (unsigned)G.tx_bytes, G.smem, G.split[0],
                    (long long)G.split[G.grid], F, mono, G.slots);
      }
    }
  }
  // the two-phase CG kernel (float64 path, and the float32 fallback): one geometry per (mesh, Np)
  for (auto& m : meshes) {
    Grid g{};
    g.nx = m[0]; g.ny = m[1]; g.nz = m[2];
    g.Px = g.nx + 1; g.Py = g.ny + 1; g.Pz = g.nz + 1;
    g.G = (long long)g.Px * g.Py * g.Pz;
    g.nI = (g.nx - 1) * (g.ny - 1) * (g.nz - 1);
    for (int Np = 4; Np <= 256; Np += 4)
      for (int sz = 4; sz <= 8; sz += 4) {
        K1Geom G{};
        int bw = 0;
        cudaError_t e = sz == 4 ? cg_plan_geometry<float>(g, Np, 152, &G, &bw)
                                : cg_plan_geometry<double>(g, Np, 152, &G, &bw);
        std::printf("P %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %u %zu\n", g.nx, g.ny, g.nz, Np,
                    sz, (int)e, bw, G.TX, G.TY, G.DX, G.npt, G.nthr, G.G4, G.nob, G.ncx, G.ncy, G.grid, G.off_p,
                    G.off_d, G.off_w, (unsigned)G.tx_bytes, G.smem);
      }
  }
  // the constant mass stencil of the library (host-computed), for three box shapes
  const double boxes[][3] = {{0.5, 0.5, 0.5}, {0.4, 0.75, 1.3}, {2.0, 0.125, 0.3}};
  for (auto& h : boxes) {
    Grid g{};
    g.nx = g.ny = g.nz = 6;
    g.hx = h[0]; g.hy = h[1]; g.hz = h[2];
    Weights27 w{};
    mass_weights(g, &w);
    std::printf("M %.17g %.17g %.17g", h[0], h[1], h[2]);
    for (int o = 0; o < 27; ++o) std::printf(" %.17g", w.w[o]);
    std::printf("\n");
  }
  return 0;
}
'''

FIELDS = ("nx ny nz Np TX TY DX ncx ncy nob grid G4 npt nthr off_p off_s off_d off_w slot tx smem "
          "s0 sN F mono maxcost").split()
TWO = "nx ny nz Np sz rc bw TX TY DX npt nthr G4 nob ncx ncy grid off_p off_d off_w tx smem".split()
KWS = 28  # packed operator weights per node (27 + one pad)


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
        src, exe = os.path.join(d, "plan.cu"), os.path.join(d, "plan")
        with open(src, "w") as f:
            f.write(SRC)
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-I", CSRC,
                        "-I", os.path.join(ROOT, "include"), src, "-o", exe, "-L", LIBDIR, "-lparo",
                        "-Xlinker", "-rpath=" + LIBDIR, "-lcuda"], check=True, capture_output=True, timeout=600)
        out = subprocess.run([exe], capture_output=True, text=True, check=True, timeout=600).stdout
    counts, geoms, mass, two = {}, [], [], []
    counts2, geoms2 = {}, []
    for line in out.splitlines():
        t = line.split()
        if t[0] == "n":
            counts2[tuple(int(v) for v in t[1:5])] = int(t[5])
        elif t[0] == "C":
            geoms2.append(dict(zip(FIELDS, (int(v) for v in t[1:]))))
        elif t[0] == "P":
            two.append(dict(zip(TWO, (int(v) for v in t[1:]))))
        elif t[0] == "M":
            mass.append(([float(v) for v in t[1:4]], [float(v) for v in t[4:]]))
        elif t[0] == "N":
            counts[tuple(int(v) for v in t[1:5])] = int(t[5])
        elif t[0] == "G":
            geoms.append(dict(zip(FIELDS, (int(v) for v in t[1:]))))
    return counts, geoms, mass, two, counts2, geoms2


def test_every_mesh_and_orbital_count_has_a_geometry(plans):
    counts, geoms = plans[0], plans[1]
    assert len(counts) == 10 * 64
    assert all(n >= 1 for n in counts.values()), [k for k, n in counts.items() if n == 0]
    assert len(geoms) == sum(counts.values())


def test_tma_boxes_and_slots_obey_the_hardware_rules(plans):
    for G in plans[1]:
        bw = 4 * G["G4"]
        # boxes: [bw][TY+2][TX+2] of r, w, s; [TY+2][DX] of D^-1; [TY][TX][28] of the weights
        for dim in (bw, G["TX"] + 2, G["TY"] + 2, G["DX"], G["TX"], G["TY"], KWS):
            assert 1 <= dim <= 256, G
        # inner extents (float32) and start coordinates (orbital block offsets, column origins) on 16 bytes
        assert (4 * bw) % 16 == 0 and (4 * G["DX"]) % 16 == 0 and (4 * KWS) % 16 == 0, G
        assert G["TX"] % 4 == 0, G
        vec = (G["TX"] + 2) * (G["TY"] + 2) * bw * 4
        dv = G["DX"] * (G["TY"] + 2) * 4
        wv = KWS * G["TX"] * G["TY"] * 4
        assert G["tx"] == 3 * vec + dv + wv and G["tx"] < 2 ** 20, G
        offs = (0, G["off_p"], G["off_s"], G["off_d"], G["off_w"], G["slot"])
        assert all(o % 128 == 0 for o in offs), G
        sizes = (vec, vec, vec, dv, wv)
        assert all(offs[i + 1] - offs[i] >= sizes[i] for i in range(5)), G


def test_launch_shape_fits_one_cta_per_sm_limits(plans):
    for G in plans[1]:
        assert G["TX"] * G["TY"] == G["nthr"] * G["npt"], G
        assert G["nthr"] * G["G4"] <= 1024, G
        assert G["smem"] <= 227 * 1024, G
        assert 1 <= G["grid"] <= 512, G


def test_tiles_blocks_and_split_cover_the_work_once(plans):
    for G in plans[1]:
        assert (G["ncx"] - 1) * G["TX"] < G["nx"] - 1 <= G["ncx"] * G["TX"], G
        assert (G["ncy"] - 1) * G["TY"] < G["ny"] - 1 <= G["ncy"] * G["TY"], G
        bw = 4 * G["G4"]
        assert (G["nob"] - 1) * bw < G["Np"] <= G["nob"] * bw, G
        assert G["s0"] == 0 and G["sN"] == G["F"] and G["mono"] == 1, G
        # balanced: no CTA carries much more than an equal share of planes and halo planes
        nzo = G["nz"] - 1
        fair = (G["F"] + 2 * (G["F"] // nzo)) / G["grid"]
        assert G["maxcost"] <= fair + nzo + 4, G


def test_library_mass_stencil_equals_the_oracle_mass_matrix(plans):
    # the 27 weights the library applies for M (computed on the host at handle
    # creation) against a row of the oracle's element-by-element assembled M
    import numpy as np

    from oracle import paro as O

    mass = plans[2]
    assert len(mass) == 3
    for h, w in mass:
        mesh = O.Mesh((6, 6, 6), (0.0, 0.0, 0.0), tuple(6 * v for v in h))
        M = O.assemble(mesh, np.zeros(8 * 216), 0.0).M.tocsr()
        row = mesh.interior_index(3, 3, 3)
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    ref = M[row, mesh.interior_index(3 + dx, 3 + dy, 3 + dz)]
                    got = w[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)]
                    assert abs(got - ref) <= 1e-15 * abs(ref), (h, dx, dy, dz, got, ref)


def test_two_phase_kernel_geometry_obeys_the_same_rules(plans):
    two = plans[3]
    assert len(two) == 10 * 64 * 2
    for G in two:
        assert G["rc"] == 0, G
        sz, bw = G["sz"], G["bw"]
        assert bw == 4 * G["G4"] and (G["nob"] - 1) * bw < G["Np"] <= G["nob"] * bw, G
        for dim in (bw, G["TX"] + 2, G["TY"] + 2, G["DX"], G["TX"], G["TY"], KWS):
            assert 1 <= dim <= 256, G
        assert (sz * bw) % 16 == 0 and (sz * G["DX"]) % 16 == 0 and (sz * KWS) % 16 == 0 and G["TX"] % 4 == 0, G
        vec = (G["TX"] + 2) * (G["TY"] + 2) * bw * sz
        dv = G["DX"] * (G["TY"] + 2) * sz
        wv = KWS * G["TX"] * G["TY"] * sz
        assert G["tx"] == 2 * vec + dv + wv and G["tx"] < 2 ** 20, G
        offs = (0, G["off_p"], G["off_d"], G["off_w"])
        assert all(o % 128 == 0 for o in offs) and all(offs[i + 1] - offs[i] >= (vec, vec, dv)[i] for i in range(3)), G
        assert G["TX"] * G["TY"] == G["nthr"] * G["npt"] and G["nthr"] * G["G4"] <= 1024, G
        assert G["smem"] <= 227 * 1024 and G["grid"] >= 1, G
        assert (G["ncx"] - 1) * G["TX"] < G["nx"] - 1 <= G["ncx"] * G["TX"], G
        assert (G["ncy"] - 1) * G["TY"] < G["ny"] - 1 <= G["ncy"] * G["TY"], G


def test_single_pass_kernel_geometry(plans):
    # group-major vectors: each active group of four orbitals is one TMA box of
    # [TY+2][4 (TX+2)] floats per plane (16 B per node, a row contiguous)
    counts2, geoms2 = plans[4], plans[5]
    assert len(counts2) == 10 * 64 and all(n >= 1 for n in counts2.values())
    assert len(geoms2) == sum(counts2.values())
    static = 64  # the kernel's static shared memory (a few ints)
    for G in geoms2:
        bw = 4 * G["G4"]
        assert 1 <= G["G4"] <= 8, G
        for dim in (4 * (G["TX"] + 2), G["TY"] + 2, G["DX"], G["TX"], G["TY"], KWS):
            assert 1 <= dim <= 256, G
        # inner extents: 16 (TX+2), 4 DX, 4 * 28 bytes; column origins 16 tx TX bytes
        assert (4 * G["DX"]) % 16 == 0 and G["TX"] % 4 == 0 and G["TX"] * G["TY"] % 32 == 0, G
        box = (G["TX"] + 2) * (G["TY"] + 2) * 16
        stride = (box + 127) // 128 * 128  # every group's box starts 128-byte aligned (TMA destination)
        vec = G["G4"] * stride
        dv = G["DX"] * (G["TY"] + 2) * 4
        wv = KWS * G["TX"] * G["TY"] * 4
        assert G["tx"] == 3 * G["G4"] * box + dv + wv and G["tx"] < 2 ** 20, G
        offs = (0, G["off_p"], G["off_s"], G["off_d"], G["off_w"], G["slot"])
        assert all(o % 128 == 0 for o in offs), G
        assert all(offs[i + 1] - offs[i] >= (vec, vec, vec, dv, wv)[i] for i in range(5)), G
        # one or two nodes (stacked in y) per consumer thread, whole warps per group
        # slot; one producer warp more (512 threads at most, 384 with two nodes a thread)
        assert G["npt"] in (1, 2) and G["nthr"] * G["npt"] == G["TX"] * G["TY"] and G["TY"] % G["npt"] == 0, G
        nt = G["nthr"] * G["G4"] + 32
        assert nt <= (512 if G["npt"] == 1 else 384), G
        assert (nt - 32) % 32 == 0 and G["nthr"] % 32 == 0 and G["smem"] + static <= 227 * 1024, G
        # 3 to 6 ring slots (two mbarriers each in the first 128 bytes); sums [5 Np],
        # state (6 Np words), the flush's per-warp sums (5 x 4 per consumer warp) and
        # an owner's five totals
        slots = G["maxcost"]
        assert 3 <= slots <= 6 and 2 * 6 * 8 <= 128, G
        red = 5 * G["Np"] + 5 * G["Np"] + (nt - 32) // 32 * 20 + 8
        # float32 alpha, beta [Np]; group flags [Np/4]; per block counts and lists; 8 B of alignment
        small = (2 * G["Np"] + G["Np"] // 4 + G["nob"] + G["nob"] * G["G4"]) * 4 + 8
        assert G["smem"] == 128 + slots * G["slot"] + 8 * red + small, G
        assert 1 <= G["grid"] <= 152, G
        assert (G["ncx"] - 1) * G["TX"] < G["nx"] - 1 <= G["ncx"] * G["TX"], G
        assert (G["ncy"] - 1) * G["TY"] < G["ny"] - 1 <= G["ncy"] * G["TY"], G
        assert (G["nob"] - 1) * bw < G["Np"] <= G["nob"] * bw, G
        assert G["s0"] == 0 and G["sN"] == G["F"] and G["mono"] == 1, G
