"""The Python binding's host side, on the CPU.

* Every ctypes structure mirrors its C struct in include/qfca.h: the same size
  and the same offset for every field, as the C compiler lays them out (a
  mismatch would make every call read the wrong bytes).
* The binding refuses wrong arguments before anything reaches the library:
  host tensors where device tensors are required, wrong dtypes, non-contiguous
  tensors, wrong ranks, and mismatched per-image lists.
"""
import ctypes
import os
import subprocess

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# ctypes class in the binding -> C typedef in include/qfca.h
MIRRORS = {"Fmap": "qfca_fmap", "Basis": "qfca_basis", "BatchOutputs": "qfca_batch_outputs", "Image": "qfca_image",
           "AssocImage": "qfca_assoc_image", "MedianImage": "qfca_median_image",
           "ServeConfig": "qfca_serve_config", "Request": "qfca_request", "Result": "qfca_result"}


@pytest.fixture(scope="module")
def q():
    from paper_2510_15602_gb300 import qfca
    return qfca


@pytest.fixture(scope="module")
def c_layout(q, tmp_path_factory):
    """{typedef: (sizeof, {field: offsetof})} from a C program compiled against the header."""
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "qfca.h"', "int main(void) {"]
    for cls, ty in MIRRORS.items():
        lines.append(f'    printf("{ty} size %zu\\n", sizeof({ty}));')
        for name, _ in getattr(q, cls)._fields_:
            lines.append(f'    printf("{ty} {name} %zu\\n", offsetof({ty}, {name}));')
    lines += ["    return 0;", "}"]
    d = tmp_path_factory.mktemp("layout")
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    out = {}
    for ln in subprocess.check_output([str(exe)], text=True).splitlines():
        ty, field, v = ln.split()
        size, offs = out.setdefault(ty, [None, {}])
        if field == "size":
            out[ty][0] = int(v)
        else:
            offs[field] = int(v)
    return out


@pytest.mark.parametrize("cls", sorted(MIRRORS))
def test_ctypes_mirror_matches_c_layout(q, c_layout, cls):
    ty = MIRRORS[cls]
    size, offs = c_layout[ty]
    S = getattr(q, cls)
    assert ctypes.sizeof(S) == size, (cls, ctypes.sizeof(S), size)
    for name, _ in S._fields_:
        assert getattr(S, name).offset == offs[name], (cls, name)


def test_host_tensors_rejected(q):
    X = torch.zeros(4, 8, 8)
    with pytest.raises(ValueError, match="CUDA"):
        q.fit_pca(X, 2)
    with pytest.raises(ValueError, match="CUDA"):
        q.covariance(X)
    with pytest.raises(ValueError, match="CUDA"):
        q.quantize(X, (torch.zeros(4, dtype=torch.float64), torch.zeros(4, 2, dtype=torch.float64)), 16)
    with pytest.raises(ValueError, match="CUDA"):
        q.score(torch.zeros(2, 8, 16, dtype=torch.uint8), 8, 16, 1, torch.zeros(2, 16, dtype=torch.int32), 64)
    with pytest.raises(ValueError, match="CUDA"):
        q.score_assoc(torch.zeros(2, 8, 16, dtype=torch.uint8), 8, 16, 1, torch.zeros(2, 16, dtype=torch.int32), 64)
    with pytest.raises(ValueError, match="CUDA"):
        q.median_reference(torch.zeros(2, 8, 16, dtype=torch.uint8), 8, 16, 1)
    with pytest.raises(ValueError, match="CUDA"):
        q.batch_run(torch.zeros(2, 4, 8, 8), 2, 16, 1)
    with pytest.raises(ValueError, match="CUDA"):
        q.batch_run_plus(torch.zeros(2, 4, 8, 8), 2, 16, 1)
    with pytest.raises(ValueError, match="CUDA"):
        q.quantize_residual(X, (torch.zeros(4, dtype=torch.float64), torch.zeros(4, 2, dtype=torch.float64)), 16)


def test_wrong_dtype_layout_and_rank_rejected(q, monkeypatch):
    # pretend every tensor is on the device, so the dtype, contiguity and rank checks are reached
    monkeypatch.setattr(torch.Tensor, "is_cuda", property(lambda self: True))
    with pytest.raises(ValueError, match="float32"):
        q.fit_pca(torch.zeros(4, 8, 8, dtype=torch.float64), 2)
    with pytest.raises(ValueError, match="contiguous"):
        q.fit_pca(torch.zeros(8, 8, 4).permute(2, 0, 1), 2)
    with pytest.raises(ValueError, match="3-D"):
        q.fit_pca(torch.zeros(4, 64), 2)
    with pytest.raises(ValueError, match="uint8"):
        q.score(torch.zeros(2, 8, 16, dtype=torch.int32), 8, 16, 1, torch.zeros(2, 16, dtype=torch.int32), 64)
    with pytest.raises(ValueError, match="ref_hist"):
        q.score(torch.zeros(2, 8, 16, dtype=torch.uint8), 8, 16, 1, torch.zeros(2, 16, dtype=torch.float32), 64)
    with pytest.raises(ValueError, match=r"\[nimg, C, H, W\]"):
        q.batch_run(torch.zeros(4, 8, 8), 2, 16, 1)
    with pytest.raises(ValueError, match="float64"):
        q.quantize(torch.zeros(4, 8, 8), (torch.zeros(4, dtype=torch.float32), torch.zeros(4, 2)), 16)


def test_per_image_lists_must_agree(q, monkeypatch):
    monkeypatch.setattr(torch.Tensor, "is_cuda", property(lambda self: True))
    b = torch.zeros(2, 8, 16, dtype=torch.uint8)
    R = torch.zeros(2, 16, dtype=torch.int32)
    with pytest.raises(ValueError, match="one width"):
        q.score_assoc_batch([b, b], [8], [1, 1], 16, [R, R], [64, 64])
    with pytest.raises(ValueError, match="one width and radius"):
        q.median_reference_batch([b, b], [8, 8], [1], 16)
    with pytest.raises(ValueError, match="one radius per image"):
        q.score_batch([torch.zeros(4, 8, 8)], [], 2, 16)


def test_shape_checks_come_before_the_context(q, monkeypatch):
    # with every tensor passing as a device tensor, a malformed call must fail on its
    # shape before any context (and so any CUDA initialisation) is created
    monkeypatch.setattr(torch.Tensor, "is_cuda", property(lambda self: True))
    monkeypatch.setattr(q, "default_context", lambda *a, **k: pytest.fail("context created before the shape check"))
    with pytest.raises(ValueError, match="3-D"):
        q.covariance(torch.zeros(4, 64))
    with pytest.raises(ValueError, match="3-D"):
        q.quantize(torch.zeros(4, 64), (torch.zeros(4, dtype=torch.float64), torch.zeros(4, 2, dtype=torch.float64)), 16)
    with pytest.raises(ValueError, match="channel count"):
        q.score_batch([torch.zeros(4, 8, 8), torch.zeros(5, 8, 8)], [1, 1], 2, 16)
