"""The C ABI's input and output forms give identical results: relevance as FP32 or FP64 host arrays,
host or CUDA torch tensors, rows padded to a larger leading dimension (a view of a wider array,
passed as ld without a copy) and BF16 as raw bits or a torch tensor; policies and gradients written
to host arrays or to CUDA tensors. Every form imports the same FP32 (or BF16) values, so the
trajectories must agree bit for bit."""
import numpy as np
import pytest

from gpu_util import require_gpu
from paper_2406_10262_gb300 import fairrank as fr
from paper_2406_10262_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    require_gpu()
    import torch as t
    return t


def run(U, I, K, param, r, steps=3, **kw):
    g = fr.FairRank(U, I, K, param=param, sinkhorn_iters=20, **kw)
    g.set_relevance(r)
    g.set_exposure(synth.dcg_exposure(K))
    F = g.step(steps)
    out = (F, g.policy(), g.impacts()[0])
    g.close()
    return out


@pytest.mark.parametrize("param", [fr.PARAM_FULL_C, fr.PARAM_ITEM])
def test_relevance_input_forms_agree(torch, param):
    U, I, K = 37, 300, 10
    r32 = synth.relevance_lowrank(U, I, seed=21).astype(np.float32)
    wide = np.zeros((U, I + 19), np.float32)  # rows padded to ld = 319 elements
    wide[:, :I] = r32
    wide[:, I:] = 7.0                         # padding the library must not read
    wide_t = torch.from_numpy(wide).cuda()
    forms = {
        "f64": r32.astype(np.float64),
        "view": wide[:, :I],
        "torch_cpu": torch.from_numpy(r32.copy()),
        "torch_cuda": torch.from_numpy(r32.copy()).cuda(),
        "torch_cuda_view": wide_t[:, :I],
    }
    assert not forms["view"].flags["C_CONTIGUOUS"] and forms["view"].strides[0] == 4 * (I + 19)
    F0, X0, imp0 = run(U, I, K, param, r32)
    for name, r in forms.items():
        F, X, imp = run(U, I, K, param, r)
        np.testing.assert_array_equal(F, F0, err_msg=name)
        np.testing.assert_array_equal(X, X0, err_msg=name)
        np.testing.assert_array_equal(imp, imp0, err_msg=name)


def test_bf16_bits_and_torch_bfloat16_agree(torch):
    U, I, K = 20, 200, 5
    r = synth.relevance_lowrank(U, I, seed=22).astype(np.float32)
    bits = synth.to_bf16_bits(r)
    F0, X0, _ = run(U, I, K, fr.PARAM_ITEM, bits, rel_dtype=fr.BF16)
    rt = torch.from_numpy(bits.view(np.int16).copy()).view(torch.bfloat16).cuda()
    F1, X1, _ = run(U, I, K, fr.PARAM_ITEM, rt, rel_dtype=fr.BF16)
    np.testing.assert_array_equal(F1, F0)
    np.testing.assert_array_equal(X1, X0)


@pytest.mark.parametrize("param", [fr.PARAM_FULL_C, fr.PARAM_ITEM])
def test_outputs_to_device_buffers(torch, param):
    U, I, K = 11, 150, 10
    g = fr.FairRank(U, I, K, param=param, sinkhorn_iters=20)
    g.set_relevance(synth.relevance_lowrank(U, I, seed=23).astype(np.float32))
    g.set_exposure(synth.dcg_exposure(K))
    g.step(2)
    X = g.policy(2, 5)
    Xd = torch.zeros((5, I, fr.num_cols(I, K)), dtype=torch.float32, device="cuda")
    g.policy(2, 5, out=Xd)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(Xd.cpu().numpy(), X)
    want_dr = param == fr.PARAM_ITEM
    dh = g.grad(want_dr=want_dr)
    dd = g.grad(want_dr=want_dr, device=True)
    torch.cuda.synchronize()
    dh, dd = (dh, dd) if want_dr else ((dh,), (dd,))
    for a, b in zip(dh, dd):
        np.testing.assert_array_equal(b.cpu().numpy(), a)
    g.close()


def test_batch_relevance_forms_agree(torch):
    sizes = [(9, 120, 10), (14, 300, 5)]
    rs = [synth.relevance_lowrank(U, I, seed=30 + j).astype(np.float32)
          for j, (U, I, K) in enumerate(sizes)]

    def batch(forms):
        b = fr.FairRankBatch(sizes, sinkhorn_iters=20)
        for j, ((U, I, K), r) in enumerate(zip(sizes, forms)):
            b.set_relevance(j, r)
            b.set_exposure(j, synth.dcg_exposure(K))
        F = b.step(3)
        b.close()
        return F

    F0 = batch(rs)
    wide = [np.pad(r, ((0, 0), (0, 13)), constant_values=5.0) for r in rs]
    F1 = batch([torch.from_numpy(rs[0].copy()).cuda(), wide[1][:, :sizes[1][1]]])
    np.testing.assert_array_equal(F1, F0)


def test_relevance_leading_dimension_below_items_is_rejected(torch):
    g = fr.FairRank(4, 30, 5)
    r = np.ones((4, 30), np.float32)
    with pytest.raises(fr.FairRankError) as ei:
        g.set_relevance(r[:, ::2])  # 15 columns (copied to a dense array): ld 15 < 30 items
    assert ei.value.status == 1  # FR_EINVAL
    g.close()
