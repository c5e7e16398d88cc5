"""The autotuner's cache file (OCT_HYDRO_TUNE_CACHE): a tuning result is
stored once and applied on the next autotune without trial launches."""
import numpy as np
import pytest

import oracle
from paper_2210_06439_gb300 import inputs
from tests.helpers import e3s, field_errors, oracle_filled

pytestmark = pytest.mark.gpu


def test_cache_stores_and_applies(tmp_path, monkeypatch):
    import torch
    from paper_2210_06439_gb300 import binding
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("OCT_HYDRO_TUNE_CACHE", str(path))
    p = oracle_filled(inputs.periodic_box(nsub=2))
    U = torch.from_numpy(p.U).cuda()
    H = binding.Hydro.from_problem(p)
    H.autotune(U)
    lines = path.read_text().split("\n")
    lines = [ln for ln in lines if ln]
    assert len(lines) == 1
    key, mode, use = lines[0].split()
    assert "|f0|nf11|e8x8," in key
    assert H.launch_info()[:2] == (int(mode), int(use))
    H.close()
    # a stored result for the same key is applied as it is, without timing
    path.write_text(f"{key} 0 1\n")
    H = binding.Hydro.from_problem(p)
    H.autotune(U)
    assert H.launch_info()[:2] == (0, 1)
    assert len([ln for ln in path.read_text().split("\n") if ln]) == 1
    d = torch.zeros(H.rhs_len, dtype=torch.float64, device="cuda")
    H.rhs(U, d)
    torch.cuda.synchronize()
    d_o, _, _ = oracle.rhs(p.edge, p.off, p.dx, p.nf, p.U)
    assert np.all(field_errors(d.cpu().numpy(), d_o, p.nf, e3s(p)) <= 1e-12)
    # another form has another key
    H.set_params(precision=1)
    H.autotune(U)
    assert len([ln for ln in path.read_text().split("\n") if ln]) == 2
