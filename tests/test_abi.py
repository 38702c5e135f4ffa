"""The C-ABI library loads, exports every function include/grbk.h declares, and
the Python binding's ctypes structs have the C layout (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2408_05444_gb300 as g
from paper_2408_05444_gb300 import build as gbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "grbk.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(grbk_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def built():
    return gbuild.build()


def test_every_declared_symbol_is_exported(built):
    names = declared_functions()
    assert len(names) >= 12
    L = ctypes.CDLL(built)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert set(names) == set(g.EXPORTS)


def test_strerror_without_gpu(built):
    assert g.grbk_strerror(g.GRBK_EINVAL) == "invalid argument"
    assert g.grbk_strerror(99) == "unknown status"


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "grbk.h"
int main(void) {
  printf("%zu %zu %zu\\n", sizeof(grbk_mat), sizeof(grbk_opts), sizeof(grbk_result));
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", offsetof(grbk_opts, alpha), offsetof(grbk_opts, x_ref),
         offsetof(grbk_opts, trace_len), offsetof(grbk_opts, stream), offsetof(grbk_opts, check_every),
         offsetof(grbk_result, status), offsetof(grbk_result, x0_rejected), offsetof(grbk_opts, use_gram),
         offsetof(grbk_opts, alphas), offsetof(grbk_opts, extended), offsetof(grbk_opts, tune),
         offsetof(grbk_opts, deferred), offsetof(grbk_result, deferred));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split()
    sizes = list(map(int, out[:3]))
    offs = list(map(int, out[3:]))
    assert sizes == [ctypes.sizeof(g.grbk_mat), ctypes.sizeof(g.grbk_opts), ctypes.sizeof(g.grbk_result)]
    assert offs == [g.grbk_opts.alpha.offset, g.grbk_opts.x_ref.offset, g.grbk_opts.trace_len.offset,
                    g.grbk_opts.stream.offset, g.grbk_opts.check_every.offset, g.grbk_result.status.offset,
                    g.grbk_result.x0_rejected.offset, g.grbk_opts.use_gram.offset, g.grbk_opts.alphas.offset,
                    g.grbk_opts.extended.offset, g.grbk_opts.tune.offset, g.grbk_opts.deferred.offset,
                    g.grbk_result.deferred.offset]


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(g, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(g, "_lib", None)
    with pytest.raises(RuntimeError):
        g.lib()


def test_option_marshalling_without_gpu(built):
    """The binding's keyword options land in the grbk_opts fields the header
    declares, and the library's defaults are the documented ones."""
    o = g.grbk_default_opts()
    assert (o.precision, o.refresh_T, o.alpha, o.stop_kind, o.split_terms) == (g.GRBK_F64, 0, 0.0, 0, 2)
    assert (o.use_gram, o.form, o.rank_tol, o.band_limit) == (0, g.GRBK_FORM_FULL, 0.0, 0)
    o, keep = g._make_opts(None, precision="f32", refresh_T=64, split_terms=3, use_gram=False, form="rowspace",
                           rank_tol=1e-9, band_limit=-1, stop_kind="relres", check_every=128, grid_ctas=7,
                           trace_len=5)
    assert (o.precision, o.refresh_T, o.split_terms, o.use_gram) == (g.GRBK_F32, 64, 3, -1)
    assert (o.form, o.rank_tol, o.band_limit) == (g.GRBK_FORM_ROWSPACE, 1e-9, -1)
    assert (o.stop_kind, o.check_every, o.grid_ctas, o.trace_len) == (g.GRBK_STOP_RELRES, 128, 7, 5)
    assert keep.rows.shape == (5,) and keep.S.shape == (5,)
    o2, _ = g._make_opts(None, use_gram=True)
    assert o2.use_gram == 1
    assert not o2.alphas
    o3, keep3 = g._make_opts(None, alphas=[0.5, 0.25])
    assert (o3.alphas[0], o3.alphas[1]) == (0.5, 0.25) and keep3.alphas.dtype.name == "float64"


def test_matrix_descriptors_are_checked_before_the_library():
    """The library trusts (pointer, rows, cols, row stride); views it cannot
    read in that form are refused in Python, with no library call."""
    import numpy as np
    import torch
    a = np.arange(60, dtype=np.float64).reshape(6, 10)
    d = g.mat(a)
    assert (d.rows, d.cols, d.ld, d.dtype, d.on_device) == (6, 10, 10, g.GRBK_DT_F64, 0)
    d = g.mat(a[1:, :4])  # row slice of wider rows: row stride stays 10
    assert (d.rows, d.cols, d.ld) == (5, 4, 10) and d.ptr == a[1:].ctypes.data
    assert g.mat(a[2:3, :]).ld == 10
    for bad in (np.flipud(a), np.broadcast_to(a[0], (6, 10)), a.T, a[:, ::2]):
        with pytest.raises(ValueError):
            g.mat(bad)
    with pytest.raises(TypeError):
        g.mat(a.astype(np.int32))
    with pytest.raises(TypeError):
        g.mat(a.astype(">f8"))
    with pytest.raises(ValueError):
        g.mat(a[0])
    ro = a.copy()
    ro.flags.writeable = False
    g.mat(ro)
    with pytest.raises(ValueError):
        g.mat(ro, out=True)
    with pytest.raises(TypeError):
        g.mat(a.tolist())
    t = torch.zeros(4, 6, dtype=torch.float32)
    d = g.mat(t)
    assert (d.rows, d.cols, d.ld, d.dtype) == (4, 6, 6, g.GRBK_DT_F32)
    assert g.mat(torch.zeros(4, 9)[:, :6]).ld == 9
    for bad in (torch.zeros(1, 6).expand(4, 6), torch.zeros(6, 4).t(), torch.zeros(4, 6, 2)):
        with pytest.raises(ValueError):
            g.mat(bad)
    with pytest.raises(TypeError):
        g.mat(torch.zeros(4, 6, dtype=torch.int32))


def test_device_only_entry_points_check_their_tensors():
    """The no-allocation solver and the U-Net entry points take contiguous FP32
    CUDA tensors of matching shapes; anything else is refused in Python."""
    import torch
    A, B, C, X = torch.zeros(8, 4), torch.zeros(3, 5), torch.zeros(8, 5), torch.zeros(4, 3)
    with pytest.raises(ValueError):  # host tensors
        g.grbk_solve_small_noalloc(A, B, C, X)
    with pytest.raises(TypeError):
        g.grbk_solve_small_noalloc(A.double(), B, C, X)
    net = g.UNetHandle(None, 4)
    with pytest.raises(ValueError):
        g.grbk_unet_forward(net, torch.zeros(2, 16, 16), torch.zeros(2, 16, 16))
    with pytest.raises(TypeError):
        g.grbk_unet_train_step(net, torch.zeros(2, 16, 16, dtype=torch.int32), torch.zeros(2, 16, 16), 1e-3)
