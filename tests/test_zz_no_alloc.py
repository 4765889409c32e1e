"""rf_nll_grad_noalloc: the NLL + gradient pass for callers that cannot
allocate device memory while they run (its scratch is a static device array
inside the library).  Checked through the C ABI against the allocating entry
point rf_nll_grad on two calls in a row, with the tolerances of the other
parity tests, for the three kinds of event program (float-float decay shape
on an FP64 column, the generic FP64 interpreter, the three-observable
float-float shape on FP32 columns), and at the largest accepted size.  This
file is collected last on purpose."""
import numpy as np
import pytest

from paper_2003_12861_gb300 import _lib as L
from paper_2003_12861_gb300 import api
from paper_2003_12861_gb300 import workloads as W

from helpers import GRAD_RTOL, NLL_RTOL

pytestmark = pytest.mark.gpu

CASES = [("decay_model", W.DECAY_TRUE, False), ("decay_generic_model", W.DECAY_GENERIC_TRUE, False),
         ("prod3_model", W.PROD3_TRUE, True)]


@pytest.mark.parametrize("which,true,f32", CASES)
def test_noalloc_matches_allocating_entry_point(oracle_mod, which, true, f32):
    import torch

    spec = W.model_for(which)
    om = oracle_mod.Model(spec.nodes, spec.root)
    n = 5 * 4096 + 1234
    cols = om.generate(true, 4242, 0, 0, n)
    if f32:
        cols = [c.astype(np.float32) for c in cols]
    m = api.Model.from_spec(spec)
    d = api.Data.upload(m, cols, f32=[f32] * spec.n_obs)
    dcol = [torch.from_numpy(c).cuda() for c in cols]
    P = m.n_free
    out = torch.zeros(1 + P, dtype=torch.float64, device="cuda")
    flags = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    thetas = [np.asarray(true, dtype=float), np.asarray(true) * (1 + 0.04 * np.sin(np.arange(P) + 2.0))]
    for th in thetas:  # two calls in a row share the static scratch
        ref_nll, ref_g = api.nll_grad(m, d, th)
        _, _, al, ag, _ = om.nll(th, [c.astype(np.float64) for c in cols])
        th_dev = torch.tensor(th, dtype=torch.float64, device="cuda")
        out.fill_(np.nan)
        api.nll_grad_noalloc(m, dcol, th_dev, out, flags)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert int(flags.item()) == 0
        assert abs(o[0] - ref_nll) <= NLL_RTOL * al, (o[0], ref_nll)
        assert np.all(np.abs(o[1:] - ref_g) <= GRAD_RTOL * ag), (o[1:], ref_g)


def test_noalloc_at_its_largest_size_matches_the_allocating_pass():
    """The largest dataset the static array takes (three FP32 columns of the
    product model), against the allocating asynchronous pass over the same
    borrowed columns: both run the same reduction tree, so the results agree
    to the last bit."""
    import torch

    spec = W.prod3_model()
    m = api.Model.from_spec(spec)
    n = api.noalloc_max_events(m)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(777)
    # uniform events on each observable's range (any in-range data will do)
    dcols = [lo + (hi - lo) * torch.rand(n, generator=gen, dtype=torch.float32, device="cuda")
             for lo, hi in ((5.2, 5.4), (0.0, 10.0), (-1.0, 1.0))]
    for c, (lo, hi) in zip(dcols, ((5.2, 5.4), (0.0, 10.0), (-1.0, 1.0))):
        c.clamp_(lo, np.nextafter(np.float32(hi), np.float32(lo)).item())
    d = api.Data.from_torch(m, dcols)
    P = m.n_free
    th = torch.tensor(W.PROD3_TRUE * (1 + 0.01 * np.cos(np.arange(P))), dtype=torch.float64, device="cuda")
    ref = torch.zeros(1 + P, dtype=torch.float64, device="cuda")
    rflags = torch.zeros(1, dtype=torch.int32, device="cuda")
    api.nll_grad_async(m, d, th, ref, rflags, stream=torch.cuda.current_stream())
    out = torch.zeros(1 + P, dtype=torch.float64, device="cuda")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    for _ in range(2):
        out.fill_(np.nan)
        api.nll_grad_noalloc(m, dcols, th, out, flags)
        torch.cuda.synchronize()
        assert int(flags.item()) == 0 and int(rflags.item()) == 0
        assert torch.equal(out, ref), (out, ref)


def test_noalloc_rejects_datasets_beyond_its_scratch():
    import torch

    m = api.Model.from_spec(W.decay_model())
    col = torch.zeros(1, dtype=torch.float64, device="cuda")
    th = torch.tensor(W.DECAY_TRUE, dtype=torch.float64, device="cuda")
    out = torch.zeros(7, dtype=torch.float64, device="cuda")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    n_over = api.noalloc_max_events(m) + 1

    class Big:  # one event beyond the limit; rejected on size before anything is read
        dtype = torch.float64
        is_cuda = True
        device = col.device

        def is_contiguous(self):
            return True

        def data_ptr(self):
            return col.data_ptr()

        def numel(self):
            return n_over

    with pytest.raises(L.RFError) as e:
        api.nll_grad_noalloc(m, [Big()], th, out, flags)
    assert e.value.status == L.RF_E_INVALID
    assert "static array" in str(e.value)
