"""The public device API (include/gq_device.cuh) from a user kernel (run with -m gpu).

tests/device_api_user.cu is compiled here against include/ only, into its own
shared object, as a library user would build it.  Its kernel mixes enqueuers
(from two divergent call sites) and dequeuers (retrying on EMPTY) in one launch
on a queue made by the host API; every item must come out exactly once."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest
import torch

import paper_2606_01693_gb300 as gq
import synth

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def user_lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = str(tmp_path_factory.mktemp("userlib") / "libuser.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-shared",
                    "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
                    os.path.join(HERE, "device_api_user.cu"), "-o", out], check=True, capture_output=True)
    L = ctypes.CDLL(out)
    L.user_mixed_launch.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_uint32]
    L.user_mixed_launch.restype = ctypes.c_int
    return L


@pytest.mark.parametrize("kind", gq.READY_KINDS)
@pytest.mark.parametrize("elem", [4, 8])
def test_user_kernel_mixed_exactly_once(user_lib, kind, elem):
    n = 8192                                  # 4096 enqueuers, 4096 dequeuers
    cap = (1 << 24) if kind == "ymc" else 1 << 13
    q = gq.Queue(kind, cap, elem, max_threads=n)
    view = ctypes.create_string_buffer(gq.GQ_VIEW_BYTES)
    assert gq.load().gq_device_view(q.handle, view) == 0
    i = np.arange(n // 2, dtype=np.uint64)
    vals = (i * np.uint64(2654435761) + np.uint64(12345)) % np.uint64(1 << 32)   # distinct (odd multiplier)
    if elem == 8:
        vals = (vals << np.uint64(24)) | (synth.splitmix64(5, i) >> np.uint64(40))
    d_in = torch.from_numpy(vals.view(np.int64)).cuda()
    d_out = torch.zeros(n // 2, dtype=torch.int64, device="cuda")
    d_st = torch.full((n,), -99, dtype=torch.int32, device="cuda")
    assert user_lib.user_mixed_launch(ctypes.addressof(view), d_in.data_ptr(), d_out.data_ptr(), d_st.data_ptr(), n) == 0
    assert q.sync_status() == 0
    st = d_st.cpu().numpy()
    assert (st == gq.GQ_OK).all(), np.unique(st, return_counts=True)
    got = np.sort(d_out.cpu().numpy().view(np.uint64))
    assert (got == np.sort(vals)).all()
    q.close()
