"""Host-side checks of the C-ABI (no GPU needed): the library exports every entry point that
include/hpt.h declares, and the ctypes structs of the binding match the C layout."""
import os
import re
import subprocess
import tempfile

import pytest

from paper_2606_14173_gb300 import hpt
from paper_2606_14173_gb300.scenes import PHASE_GRF as S_PHASE_GRF

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hpt.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"\b(hpt_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_14173_gb300 import build
    build.build()
    return hpt.load_library()


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(hpt.SYMBOLS) == names


def test_struct_layout_matches_header():
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "hpt.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(hpt_material), sizeof(hpt_scene_desc), sizeof(hpt_render_desc), sizeof(hpt_ctx_desc));
  printf("%zu %zu %zu %zu %zu\n", offsetof(hpt_scene_desc, tex_floats), offsetof(hpt_scene_desc, cache_res),
         offsetof(hpt_scene_desc, cache_E), offsetof(hpt_render_desc, seed), offsetof(hpt_render_desc, T));
  printf("%zu %zu\n", offsetof(hpt_render_desc, precision), offsetof(hpt_render_desc, use_cache));
  printf("%d %d %d %d\n", HPT_NCOUNTERS, HPT_NKERNELS, HPT_K_TRACE, HPT_K_ACCUM);
  printf("%zu %zu %zu %d\n", offsetof(hpt_render_desc, grf_phi), offsetof(hpt_render_desc, grf_nx),
         offsetof(hpt_render_desc, grf_ny), HPT_PHASE_GRF);
  printf("%zu %zu %zu\n", sizeof(hpt_bake_desc), offsetof(hpt_bake_desc, spp), offsetof(hpt_bake_desc, seed));
  printf("%zu\n", offsetof(hpt_render_desc, omit_obliquity));
  printf("%zu\n", offsetof(hpt_ctx_desc, max_queue));
  printf("%zu %zu %zu %d %d\n", sizeof(hpt_tuning), offsetof(hpt_tuning, band_ms), offsetof(hpt_tuning, band_path_samples),
         HPT_ERR_CANCELLED, HPT_CTX_FAIL_SERVING_WAVES);
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        exe = os.path.join(d, "p")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = subprocess.check_output([exe]).decode().split()
    import ctypes as C
    got = [C.sizeof(hpt.Material), C.sizeof(hpt.SceneDesc), C.sizeof(hpt.RenderDesc), C.sizeof(hpt.CtxDesc),
           hpt.SceneDesc.tex_floats.offset, hpt.SceneDesc.cache_res.offset, hpt.SceneDesc.cache_E.offset,
           hpt.RenderDesc.seed.offset, hpt.RenderDesc.T.offset, hpt.RenderDesc.precision.offset,
           hpt.RenderDesc.use_cache.offset, hpt.NCOUNTERS, len(hpt.KERNEL_NAMES),
           hpt.KERNEL_NAMES.index("k_trace"), hpt.KERNEL_NAMES.index("k_accum"),
           hpt.RenderDesc.grf_phi.offset, hpt.RenderDesc.grf_nx.offset, hpt.RenderDesc.grf_ny.offset, S_PHASE_GRF,
           C.sizeof(hpt.BakeDesc), hpt.BakeDesc.spp.offset, hpt.BakeDesc.seed.offset,
           hpt.RenderDesc.omit_obliquity.offset, hpt.CtxDesc.max_queue.offset,
           C.sizeof(hpt.Tuning), hpt.Tuning.band_ms.offset, hpt.Tuning.band_path_samples.offset,
           [k for k, v in hpt.STATUS_NAMES.items() if v == "CANCELLED"][0], hpt.CTX_FAIL_SERVING_WAVES]
    assert [int(x) for x in out] == got


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(RuntimeError):
        hpt._lib_save = hpt._lib
        try:
            hpt._lib = None
            hpt.load_library(str(tmp_path / "nope.so"))
        finally:
            hpt._lib = hpt._lib_save


def test_render_desc_marshalling():
    from paper_2606_14173_gb300 import scenes as S
    r = S.config2_render(seed=(5 << 32) | 7)
    d = hpt.render_desc(r, hpt.PREC_FP64)
    assert (d.W, d.H, d.n_lambda, d.K, d.spp, d.max_depth) == (1920, 1080, 3, 8, 64, 4)
    assert d.seed == (5 << 32) | 7 and d.precision == 0
    assert list(d.channel) == [0, 1, 2] and abs(d.lam[2] - 450e-9) < 1e-20
    assert hpt.out_bytes(r) == 8 * 3 * 8 * 1920 * 1080
