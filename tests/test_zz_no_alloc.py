"""rf_nll_grad_noalloc: the NLL + gradient pass for callers that cannot
allocate device memory while they run (its scratch is a static device array
inside the library).  Checked through the C ABI against the allocating entry
point rf_nll_grad on two calls in a row, with the tolerances of the other
parity tests.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2003_12861_gb300 import _lib as L
from paper_2003_12861_gb300 import api
from paper_2003_12861_gb300 import workloads as W

from helpers import GRAD_RTOL, NLL_RTOL, TRUE

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_entry_point(oracle_mod):
    import torch

    spec = W.decay_model()
    om = oracle_mod.Model(spec.nodes, spec.root)
    n = 5 * 4096 + 1234
    cols = om.generate(TRUE["decay_model"], 4242, 0, 0, n)
    m = api.Model.from_spec(spec)
    d = api.Data.upload(m, cols)
    dcol = [torch.from_numpy(cols[0]).cuda()]
    out = torch.zeros(1 + m.n_free, dtype=torch.float64, device="cuda")
    flags = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    thetas = [TRUE["decay_model"], TRUE["decay_model"] * (1 + 0.04 * np.sin(np.arange(6) + 2.0))]
    for th in thetas:  # two calls in a row share the static scratch
        ref_nll, ref_g = api.nll_grad(m, d, th)
        _, _, al, ag, _ = om.nll(th, cols)
        th_dev = torch.tensor(th, dtype=torch.float64, device="cuda")
        api.nll_grad_noalloc(m, dcol, th_dev, out, flags)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert int(flags.item()) == 0
        assert abs(o[0] - ref_nll) <= NLL_RTOL * al, (o[0], ref_nll)
        assert np.all(np.abs(o[1:] - ref_g) <= GRAD_RTOL * ag), (o[1:], ref_g)


def test_noalloc_rejects_datasets_beyond_its_scratch():
    import torch

    m = api.Model.from_spec(W.decay_model())
    col = torch.zeros(1, dtype=torch.float64, device="cuda")
    th = torch.tensor(TRUE["decay_model"], dtype=torch.float64, device="cuda")
    out = torch.zeros(7, dtype=torch.float64, device="cuda")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")

    class Big:  # claims 1e9 events; rejected on size before anything is read
        dtype = torch.float64

        def data_ptr(self):
            return col.data_ptr()

        def numel(self):
            return 1_000_000_000

    with pytest.raises(L.RFError) as e:
        api.nll_grad_noalloc(m, [Big()], th, out, flags)
    assert e.value.status == L.RF_E_INVALID
    assert "static array" in str(e.value)
