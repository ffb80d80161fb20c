"""janc_rhs_static, the right-hand side for callers that cannot allocate
device memory (for example code running inside another framework's memory
pool, where a raw cudaMalloc would bypass the pool): its result must equal
janc_rhs's on the same state bit for bit (the same kernels in the same launch
shapes), and the oracle's within the right-hand-side bar, on consecutive calls
that share the one static scratch array, one of them on a grid with dx != dy.
This file is named so that pytest collects it last."""
import numpy as np
import pytest

import oracle as orc
from paper_2504_13750_gb300 import inputs

pytestmark = pytest.mark.gpu

H2AIR = inputs.load_mechanism("h2air_synth")


def _state(nx, ny, seed, aspect=1.0):
    st = inputs.tube(H2AIR, nx, ny, perturb_seed=seed, aspect=aspect)
    rng = np.random.default_rng(seed)
    st["u"] = rng.normal(0, 150.0, (ny, nx))
    st["v"] = rng.normal(0, 150.0, (ny, nx))
    U = orc.prim_to_cons(H2AIR, st["T"], st["p"], st["u"], st["v"], st["Y"])
    return st, U


def _rel(a, b):
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(a.shape)
    return max(float(np.max(np.abs(a[k] - b[k])) / max(np.max(np.abs(b[k])), 1e-300)) for k in range(a.shape[0]))


def test_rhs_static_matches_rhs_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_13750_gb300 import build, janc

    build.build()
    mech = janc.Mechanism(H2AIR)
    stream = torch.cuda.current_stream().cuda_stream
    # two different states (different sizes, the second with dy = 1.7 dx),
    # one call each, back to back
    cases = [_state(96, 40, 1), _state(70, 52, 2, aspect=1.7)]
    refs = []
    for st, U in cases:
        g = janc.Grid.from_grid_dict(H2AIR, st["grid"], chemistry=True)
        g.set_state(U, st["T"])
        L, _, _, al = g.rhs()
        refs.append((L, al))
        g.close()
    for (st, U), (Lref, alref) in zip(cases, refs):
        gd = st["grid"]
        desc = janc.make_desc(gd["nx"], gd["ny"], gd["dx"], gd["dy"], gd["bc"], chemistry=True)
        Ud = torch.from_numpy(U).cuda()
        Td = torch.from_numpy(np.ascontiguousarray(st["T"])).cuda()
        Ld = torch.full(U.shape, float("nan"), dtype=torch.float64, device="cuda")
        ad = torch.zeros(2, dtype=torch.float64, device="cuda")
        janc.janc_rhs_static(desc, mech, Ud, Td, Ld, ad, stream)
        Ls = Ld.cpu().numpy()
        assert np.array_equal(Ls, Lref)
        assert np.array_equal(ad.cpu().numpy(), alref)
        L0, _, _, al0 = orc.rhs(H2AIR, gd, U, st["T"])
        assert _rel(Ls, L0) <= 1e-10
        assert np.max(np.abs(ad.cpu().numpy() - al0) / al0) < 1e-13
    # a grid beyond the static array is refused with a clear error (buffers of
    # the right size, so that only the scratch limit can refuse it)
    nx, ny = 2048, 1024
    big = janc.make_desc(nx, ny, 1e-5, 1e-5, [0, 0, 0, 0], chemistry=True)
    Ub = torch.zeros(12 * nx * ny, dtype=torch.float64, device="cuda")
    Tb = torch.full((nx * ny,), 300.0, dtype=torch.float64, device="cuda")
    Lb = torch.zeros_like(Ub)
    with pytest.raises(janc.JancError) as e:
        janc.janc_rhs_static(big, mech, Ub, Tb, Lb, None, stream)
    assert e.value.rc == -1 and "JANC_STATIC_SCRATCH_BYTES" in str(e.value)
