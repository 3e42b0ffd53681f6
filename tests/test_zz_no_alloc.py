"""The allocation-free histogram entry point, fpt_histogram_noalloc.

Some callers cannot allocate device memory: code running inside another
library's allocation-free region, on a stream an application is capturing
with allocation forbidden, or under an allocator that owns all device memory.
For them the library offers one histogram entry point that allocates nothing:
its scratch is a fixed array inside the library. These checks call it through
the C ABI and compare it with the context-based histogram of the same device
arrays, on two calls in a row (the shared array must be cleared between calls).
"""
import math

import numpy as np
import pytest

import workloads as W
from paper_2410_13683_gb300 import fpt

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu


def _compare(got, ref):
    assert np.array_equal(got["count"], ref["count"])
    nz = ref["count"] > 0
    np.testing.assert_allclose(got["log_sum_w"][nz], ref["log_sum_w"][nz], rtol=0, atol=1e-12)
    np.testing.assert_allclose(got["log_sum_w2"][nz], ref["log_sum_w2"][nz], rtol=0, atol=1e-12)
    np.testing.assert_allclose(got["sum_lw"], ref["sum_lw"], rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(got["pdf"], ref["pdf"], rtol=1e-11, atol=0)
    np.testing.assert_allclose(got["se_w"], ref["se_w"], rtol=1e-8, atol=1e-300)
    ok = np.isfinite(ref["pdf_ln"])
    assert np.array_equal(ok, np.isfinite(got["pdf_ln"]))
    np.testing.assert_allclose(got["pdf_ln"][ok], ref["pdf_ln"][ok], rtol=1e-9)
    np.testing.assert_allclose(got["se_jk"], ref["se_jk"], rtol=1e-7, atol=1e-300)
    for k in ("n_total", "n_passed", "n_under", "n_over", "n_capped", "n_tail"):
        assert got[k] == ref[k], k
    for k in ("N_mean", "N_mean_w", "ess_tail", "p_tail", "log_max_w"):
        assert got[k] == pytest.approx(ref[k], rel=1e-10), k


def test_noalloc_histogram_matches_the_context_histogram():
    torch = require_gpu()
    m = W.BM.model
    lo, hi, nb, tail = 3.0, 8.0, 160, 5.5
    s = torch.cuda.Stream()
    with fpt.fpt_init_model([m]) as ctx:
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_USER, 16, 1.0, -0.1, 0.2, np.full(16, W.BM_S),
                            np.zeros(16))
        for call in range(2):                                   # two calls in a row
            n = 20000 + 777 * call
            dn = torch.zeros(n, dtype=torch.int32, device="cuda")
            dl = torch.zeros(n, dtype=torch.float64, device="cuda")
            ds = torch.zeros(n, dtype=torch.uint8, device="cuda")
            st = fpt.fpt_run(ctx, [fpt.run_desc(0, n, seed=40 + call, A=0.6)],
                             [dict(nsteps=dn, logw=dl, status=ds)], stream=s)
            assert st == fpt.FPT_OK and fpt.fpt_sync(ctx) == fpt.FPT_OK
            out = torch.full((fpt.hist_out_doubles(nb),), float("nan"), dtype=torch.float64, device="cuda")
            fpt.fpt_histogram_noalloc(dn, dl, ds, m.dN, lo, hi, nb, out, N_tail=tail, stream=s)
            s.synchronize()
            raw = out.cpu().numpy()
            got = fpt.unpack_hist(raw, nb)
            # every output slot is written: the 11 scalars, then 5 reserved zeros
            assert np.all(np.isfinite(raw[10 * nb:])) and np.all(raw[10 * nb + 11:] == 0.0)
            ref = fpt.fpt_histogram_data(ctx, dn, dl, ds, m.dN, lo, hi, nb, N_tail=tail, stream=s)
            _compare(got, ref)
            assert got["n_total"] == n and got["n_tail"] > 0


def test_noalloc_histogram_rejects_sizes_beyond_its_scratch():
    torch = require_gpu()
    n = 64
    dn = torch.zeros(n, dtype=torch.int32, device="cuda")
    dl = torch.zeros(n, dtype=torch.float64, device="cuda")
    ds = torch.zeros(n, dtype=torch.uint8, device="cuda")
    out = torch.zeros(fpt.hist_out_doubles(2048), dtype=torch.float64, device="cuda")
    with pytest.raises(fpt.FptError) as e:
        fpt.fpt_histogram_noalloc(dn, dl, ds, 1e-3, 0.0, 1.0, fpt.FPT_NOALLOC_MAX_BINS + 1, out)
    assert e.value.status == fpt.FPT_E_INVALID and "1024" in str(e.value)
