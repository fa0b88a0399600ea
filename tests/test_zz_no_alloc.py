"""The allocation-free forward pass (rewl_mlp_forward_noalloc) against the
regular one (rewl_mlp_forward), through the C ABI.

rewl_mlp_forward_noalloc serves callers that must not allocate device memory
while they run (device memory owned by another allocator, or no room for
cudaMalloc's device-wide synchronisation where they call from): its
activations live in a static device array, so it only needs the parameters,
inputs and outputs the caller already has.  It launches the same kernels as
the regular forward pass on the same inputs, so two calls in a row -- with
different batches, so the second one finds the first one's leftovers in the
shared scratch -- must each equal the regular pass bit for bit, and both must
match the network's BF16-operand statement in oracle/mlp.py within the bound
of the other network tests.  The file is collected last so that, if it fails,
a run stopping at the first failure has run everything else.
"""
import numpy as np
import pytest

from oracle import mlp as M

pytestmark = pytest.mark.gpu


def _features(n, seed):
    rng = np.random.default_rng(seed)
    x = np.stack([rng.integers(0, 2, n), 16.0 / rng.choice([8, 16, 32, 64], n), rng.choice([0.30103, 1.0], n),
                  rng.uniform(-2, 2, n), rng.uniform(0, 1, n)], axis=1)
    return np.ascontiguousarray(x, np.float32)


def test_noalloc_forward_matches_regular_forward_on_two_calls():
    import torch
    from paper_1407_5140_gb300 import rewl as R

    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        net = R.Mlp(max_batch=1024, seed=21, stream=stream)
        host_params = net.get_params()
        params = torch.from_numpy(host_params).cuda()
        for call, n in enumerate((1024, 320)):
            xh = _features(n, 100 + call)
            x = torch.from_numpy(xh).cuda()
            y_ref = torch.empty(n, dtype=torch.float32, device="cuda")
            net.forward(x, y_ref)
            y = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
            R.mlp_forward_noalloc(params, x, y, stream=stream)
            stream.synchronize()
            a, b = y.cpu().numpy(), y_ref.cpu().numpy()
            assert np.array_equal(a, b), call
            yb, _, ya = M.forward_bf16(host_params.astype(np.float64), xh.astype(np.float64))
            assert np.all(np.abs(a.astype(np.float64) - yb) <= 4e-3 * ya), call
        net.close()


def test_noalloc_forward_rejects_batches_above_its_limit():
    import torch
    from paper_1407_5140_gb300 import rewl as R

    params = torch.zeros(R.N_PARAMS, dtype=torch.float32, device="cuda")
    for n in (1088, 100):
        x = torch.zeros((n, 5), dtype=torch.float32, device="cuda")
        y = torch.zeros(n, dtype=torch.float32, device="cuda")
        with pytest.raises(R.RewlError) as ei:
            R.mlp_forward_noalloc(params, x, y)
        assert ei.value.code == -1
    # malformed tensors never reach the library
    x = torch.zeros((64, 5), dtype=torch.float32, device="cuda")
    y = torch.zeros(64, dtype=torch.float32, device="cuda")
    for bad in (dict(params=params[:-1]), dict(x=x.double()), dict(y=y[:32]), dict(x=x.t().contiguous().t()),
                dict(x=x.cpu())):
        args = dict(params=params, x=x, y=y)
        args.update(bad)
        with pytest.raises(ValueError):
            R.mlp_forward_noalloc(args["params"], args["x"], args["y"])
