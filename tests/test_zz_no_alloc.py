"""fr_nsw_eval_noalloc, the entry point for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc: code whose device memory is owned by another allocator (a
framework's caching allocator, a fixed arena) and latency-critical loops in which cudaMalloc or
cudaFree would synchronise the device. fr_nsw_eval_noalloc serves them from a static device array
instead of allocating. Here it is called through the C ABI on consecutive calls with different
problems, and each result is checked against the context-based entry point fr_impacts (same costs,
cold-start solve) within the suite's tolerance; a repeated call must reproduce its first result
exactly, whatever ran in between. The file is named to be collected last.
"""
import ctypes as ct
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from gpu_util import NSW_RTOL, require_gpu, seeded_state
from paper_2406_10262_gb300 import fairrank as fr
from paper_2406_10262_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def entry():
    f = ct.CDLL(fr.LIB_PATH).fr_nsw_eval_noalloc
    vp = ct.c_void_p
    f.restype = ct.c_int32
    f.argtypes = [vp, vp, ct.c_int64, ct.POINTER(ct.c_double), ct.c_int32, ct.c_int32, ct.c_int32,
                  ct.c_double, ct.c_int32, vp, vp, vp]
    return f


def problem(U, I, K, seed):
    r = synth.relevance_lowrank(U, I, seed=seed).astype(np.float32)
    C, _, _, _ = seeded_state(U, I, K, seed=seed, scale=0.7)
    return r, C


def via_context(U, I, K, r, C, L, eps):
    g = fr.FairRank(U, I, K, warm_start=0, sinkhorn_iters=L, epsilon=eps)
    g.set_relevance(r)
    g.set_exposure(synth.dcg_exposure(K))
    g.set_state(param=C)
    imp, util, F = g.impacts()
    g.close()
    return imp, util, F


def via_noalloc(torch, U, I, K, r, C, L, eps, ld=None, pad=0.0):
    m = fr.num_cols(I, K)
    ld = ld or (I + 7) // 8 * 8
    Ck = np.full((U, m, ld), pad, np.float32)
    Ck[:, :, :I] = C.transpose(0, 2, 1)
    rk = np.full((U, ld), pad, np.float32)
    rk[:, :I] = r
    Cd = torch.from_numpy(Ck).cuda()
    rd = torch.from_numpy(rk).cuda()
    imp = torch.full((I,), -1.0, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    e = np.ascontiguousarray(synth.dcg_exposure(K))
    st = entry()(Cd.data_ptr(), rd.data_ptr(), ld, e.ctypes.data_as(ct.POINTER(ct.c_double)), U, I,
                 K, eps, L, imp.data_ptr(), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 0, fr.lib().fr_last_error(None)
    torch.cuda.synchronize()
    return imp.cpu().numpy(), out[1].item(), out[0].item()


def test_matches_fr_impacts_on_consecutive_calls(torch):
    cases = [(40, 300, 10, 50, 1.0, 1), (7, 37, 5, 20, 0.8, 2)]
    first = None
    for U, I, K, L, eps, seed in cases + cases[:1]:
        r, C = problem(U, I, K, seed)
        imp_ref, util_ref, F_ref = via_context(U, I, K, r, C, L, eps)
        imp, util, F = via_noalloc(torch, U, I, K, r, C, L, eps)
        assert abs(F - F_ref) <= NSW_RTOL * abs(F_ref)
        assert abs(util - util_ref) <= NSW_RTOL * abs(util_ref)
        np.testing.assert_allclose(imp, imp_ref, rtol=NSW_RTOL)
        if first is None:
            first = (imp, F)
        elif (U, I, K) == cases[0][:3]:
            np.testing.assert_array_equal(imp, first[0])  # nothing left over from the call between
            assert F == first[1]


@pytest.mark.parametrize("U,I,K,ld", [
    (30, 1000, 10, 2048),  # tile sweep: 1024-float column slots, a longer caller row stride
    (12, 300, 10, 512),    # register sweep: the staged tile takes the caller's stride
])
def test_row_stride_longer_than_the_items(torch, U, I, K, ld):
    """A caller's row stride ld beyond the item count (allowed: a multiple of 8, >= n_items), with
    garbage in the entries past n_items: the result equals the context's, which packs its rows at
    the item count rounded up to 8."""
    L, eps = 20, 1.0
    r, C = problem(U, I, K, 5)
    imp_ref, util_ref, F_ref = via_context(U, I, K, r, C, L, eps)
    imp, util, F = via_noalloc(torch, U, I, K, r, C, L, eps, ld=ld, pad=7.0)
    assert abs(F - F_ref) <= NSW_RTOL * abs(F_ref)
    assert abs(util - util_ref) <= NSW_RTOL * abs(util_ref)
    np.testing.assert_allclose(imp, imp_ref, rtol=NSW_RTOL)


FRESH_CASES = [
    (20, 2000, 20, 2000),  # 21-column tile sweep: about 172 KB of shared memory per block
    (12, 300, 10, 2048),   # register sweep staging its tile at the caller's stride: about 98 KB
]


def fresh_process_results():
    """Runs in a fresh process: the allocation-free entry point first, for every case, before any
    context exists (so no earlier call has raised a kernel's shared-memory limit), then the
    context-based results of the same problems. Prints both as JSON."""
    import torch
    from paper_2406_10262_gb300 import build as frbuild

    frbuild.build()
    out = []
    for U, I, K, ld in FRESH_CASES:
        r, C = problem(U, I, K, 9)
        imp, util, F = via_noalloc(torch, U, I, K, r, C, 20, 1.0, ld=ld, pad=3.0)
        out.append({"noalloc": list(map(float, imp)) + [util, F]})
    for j, (U, I, K, ld) in enumerate(FRESH_CASES):
        r, C = problem(U, I, K, 9)
        imp, util, F = via_context(U, I, K, r, C, 20, 1.0)
        out[j]["context"] = list(map(float, imp)) + [util, F]
    print("RESULT " + json.dumps(out))


def test_first_call_in_a_fresh_process_needs_no_context(torch):
    """Shapes whose kernels need more than the default 48 KB of dynamic shared memory, called
    before any context of the same kernel variant exists in the process: the entry point raises
    the kernel's limit itself (which allocates nothing) and matches fr_impacts."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([root, os.path.join(root, "tests")]))
    res = subprocess.run([sys.executable, os.path.abspath(__file__), "--fresh"], env=env,
                         capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-4000:]
    line = [l for l in res.stdout.splitlines() if l.startswith("RESULT ")][-1]
    for case in json.loads(line[len("RESULT "):]):
        na, cx = np.array(case["noalloc"]), np.array(case["context"])
        np.testing.assert_allclose(na[:-2], cx[:-2], rtol=NSW_RTOL)  # impacts
        assert abs(na[-2] - cx[-2]) <= NSW_RTOL * abs(cx[-2])        # utility
        assert abs(na[-1] - cx[-1]) <= NSW_RTOL * abs(cx[-1])        # F


def test_rejects_problems_larger_than_the_static_scratch(torch):
    small = torch.zeros(64, dtype=torch.float32, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    e = np.ones(7)
    # 600000 consumers x 8 columns of potentials alone exceed the 8 MiB array; rejected on the host
    st = entry()(small.data_ptr(), small.data_ptr(), 8, e.ctypes.data_as(ct.POINTER(ct.c_double)),
                 600000, 8, 7, 1.0, 10, out.data_ptr(), out.data_ptr(), 0)
    assert st == 7  # FR_EUNSUPPORTED
    assert b"static scratch" in fr.lib().fr_last_error(None)
    st = entry()(small.data_ptr(), small.data_ptr(), 12, e.ctypes.data_as(ct.POINTER(ct.c_double)),
                 4, 8, 7, 1.0, 10, out.data_ptr(), out.data_ptr(), 0)
    assert st == 1  # ld not a multiple of 8


if __name__ == "__main__" and "--fresh" in sys.argv:
    fresh_process_results()
