"""The one-step outcome distribution of 8-SD cells on the GPU.

10^5 independent copies of an 8-SD cell stepped in one launch (one warp per
cell): the multiplicities and volumes equal the oracle's bit for bit, and the
outcomes fall inside the exact support with the exact frequencies of the
enumeration (all 8! orders x 2^4 gamma outcomes; Sec. 2.2 Steps 1-3,
eqs. (gamma2), (coal_attr_0), (coal)) -- the chi-square of the oracle's own
pin, now on the device path.
"""
from collections import defaultdict

import numpy as np
import pytest
from scipy import stats

import oracle
import test_oracle_enumeration as E

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2101_06318_b300 import sdm  # noqa: E402


@pytest.mark.parametrize("n", [5, 8])
def test_gpu_many_small_cells_match_enumeration(n):
    xi0, v0, pmax = E.DESIGNS[n]
    dv = E._dv_for(xi0, v0, n, pmax)
    n_cells = 100000
    xi = np.tile(np.array(xi0, np.uint64), n_cells)
    v = np.tile(np.array(v0), n_cells)
    cs = (np.arange(n_cells + 1, dtype=np.int64) * n).astype(np.uint32)
    st = sdm.State(len(xi), n_cells, 1)
    st.init(xi, v[None, :], np.full(n_cells, dv), np.zeros(n_cells, np.uint8), cell_start=cs)
    st.step(E.DT, 2024 + n, 3, 1, golovin_b=E.B)
    xg, ag, _ = st.get_state()
    st.close()
    o = oracle.System(xi, v[None, :], cs, dv, 0, E.B, "prp")
    o.step(E.DT, 2024 + n, 3)
    assert np.array_equal(o.xi, xg)
    assert np.array_equal(o.attr.view(np.uint64), ag.view(np.uint64))
    exact = E.exact_distribution(xi0, v0, dv)
    observed = defaultdict(int)
    rows = zip(map(tuple, xg.reshape(n_cells, n).tolist()), map(tuple, ag[0].reshape(n_cells, n).tolist()))
    for row_x, row_v in rows:
        observed[(row_x, row_v)] += 1
    assert all(k in exact for k in observed)
    big = [k for k in exact if exact[k] * n_cells >= 5.0]
    f_exp = [exact[k] * n_cells for k in big]
    f_obs = [observed.get(k, 0) for k in big]
    if n_cells - sum(f_exp) > 1e-9:
        f_exp.append(n_cells - sum(f_exp))
        f_obs.append(n_cells - sum(f_obs))
    assert stats.chisquare(f_obs, f_exp).pvalue > 1e-4
