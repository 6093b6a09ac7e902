"""Host-side checks of the delayed sweep's shared-memory layout (del_layout in
hfq_delayed.cuh), compiled for the host by nvcc and printed by a small
harness: for both spin counts (the two-spin sweep and the G_up-only sweep of a
particle-hole symmetric bath) the regions are aligned and disjoint, each holds
what the kernel puts there, and the recompute's overlays fit inside the total.
No GPU is used."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_0801_1222_gb300", "csrc")
OUT = os.path.join(HERE, "_build", "layout_probe")
NW = 16            # warps per CTA (kDelNT / 32)
CAP = 227 * 1024 - 512
GTILE = 128 * 128 * 4

SRC = r'''
#include <cstdio>
#include "hfq_delayed.cuh"
using namespace hfq;
int main() {
  const int Ls[] = {37, 100, 160, 166, 200, 240, 320, 500, 512};
  const int Ks[] = {8, 16, 24, 32, 40, 64};
  for (int L : Ls) for (int K : Ks) for (int res = 0; res < 2; ++res) for (int gt = 0; gt < 2; ++gt)
  for (int ub = 1; ub <= 2; ++ub) for (int rf = 0; rf < 2; ++rf) for (int ns = 1; ns <= 2; ++ns) {
    if (res && gt) continue;
    const DelLayout d = del_layout(L, K, res, false, gt, ub, rf, ns);
    printf("%d %d %d %d %d %d %d  %d %d %d %d  %u %u %u %u %u %u %u %u %u %zu  %zu %zu %zu %d\n",
           L, K, res, gt, ub, rf, ns, d.ldS, d.KP, d.KS, d.ub,
           d.off_s, d.off_body, d.off_stage, d.off_G, d.off_U, d.off_W, d.off_diag, d.off_gtile,
           d.off_rf, d.bytes, del_stage_bytes(K, L, ub), rf_smem_need(L), gj_blocked_bytes(L),
           del_panel_floats(L, d.KP, ns));
  }
  return 0;
}
'''


def _rows():
    nvcc = os.environ.get("NVCC", "nvcc")
    if shutil.which(nvcc) is None:
        pytest.skip("nvcc not found")
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    src = OUT + ".cu"
    with open(src, "w") as f:
        f.write(SRC)
    subprocess.run([nvcc, "-std=c++17", "-O1", "-I", CSRC, "-o", OUT, src], check=True,
                   capture_output=True)
    out = subprocess.run([OUT], check=True, capture_output=True, text=True).stdout
    keys = ("L K res gt ub rf ns ldS KP KS dub off_s off_body off_stage off_G off_U off_W off_diag "
            "off_gtile off_rf bytes stage_need rf_need gjb_need panel").split()
    return [dict(zip(keys, map(int, line.split()))) for line in out.strip().splitlines()]


@pytest.fixture(scope="module")
def rows():
    return _rows()


def test_regions_aligned_disjoint_and_large_enough(rows):
    for d in rows:
        L, ns = d["L"], d["ns"]
        assert d["KP"] == d["K"] + 4 and d["KS"] % 16 == 0 and d["KS"] >= d["K"]
        assert d["panel"] % 4 == 0  # zeroed by 16-byte stores
        part = ns * NW * L * 4      # measurement partial sums of the kept spins
        stage = max(d["stage_need"], part)
        regions = [(d["off_s"], L), (d["off_stage"], stage)]
        if d["res"]:
            regions.append((d["off_G"], 2 * L * d["ldS"] * 4))
        regions += [(d["off_U"], d["panel"] * 4), (d["off_W"], d["panel"] * 4), (d["off_diag"], 2 * L * 4)]
        if d["gt"]:
            regions.append((d["off_gtile"], GTILE))
            assert d["off_gtile"] % 1024 == 0
        assert d["off_stage"] % 1024 == 0 and d["off_U"] % 128 == 0 and d["off_W"] % 128 == 0
        for (a, na), (b, _) in zip(regions, regions[1:]):
            assert a + na <= b, d
        end = regions[-1][0] + regions[-1][1]
        assert d["bytes"] >= end
        if d["rf"]:
            assert d["off_rf"] % 1024 == 0 and d["bytes"] >= d["off_rf"] + d["rf_need"]


def test_panels_hold_the_kept_spins(rows):
    for d in rows:
        L, KP = d["L"], d["KP"]
        if d["ns"] == 2:
            # the spin-down block starts at the padded stride, which is L KP
            # rounded up to 16 (mod 32) floats
            stride = d["panel"] - L * KP
            assert stride >= L * KP and stride % 32 == 16 and stride - L * KP < 32
        else:
            # one spin plus the 16-float offset at which the G_up-only sweep
            # starts W; the measurement's 2 L totals also live in U's region
            assert d["panel"] == L * KP + 16 and d["panel"] >= 2 * L
            # row r of W (16 floats into its region) and row r of U fall half
            # the banks apart
            assert ((d["off_W"] - d["off_U"]) // 4 + 16) % 32 == 16


def test_one_spin_layout_is_smaller_and_fits_a_deeper_delay(rows):
    by = {(d["L"], d["K"], d["res"], d["gt"], d["ub"], d["rf"], d["ns"]): d for d in rows}
    for (L, K, res, gt, ub, rf, ns), d in by.items():
        if ns == 1:
            assert d["bytes"] <= by[(L, K, res, gt, ub, rf, 2)]["bytes"]

    def fit(L, k_req, ns):
        # the library's choice for G in HBM with the TMA reduce flush and the
        # refinement: the largest k (steps of 8) that fits, two U blocks preferred
        for k in range(k_req, 7, -8):
            for ub in (2, 1):
                if (L, k, 0, 1, ub, 1, ns) in by and by[(L, k, 0, 1, ub, 1, ns)]["bytes"] <= CAP:
                    return k, ub
        return None

    assert fit(500, 64, 2) == (8, 2)
    assert fit(500, 64, 1) == (24, 1)
    assert fit(320, 64, 2) == (16, 2)
    assert fit(320, 40, 1) == (40, 1)
    assert fit(240, 16, 1) == (16, 2)
