"""saq_kernel_timing / saq_kernel_times: every launch of an encode is timed on
its own stream and attributed to its kind."""
import pytest
import torch

import paper_2509_12086_gb300 as P
from paper_2509_12086_gb300 import synth

pytestmark = pytest.mark.gpu


def test_kernel_times_cover_the_encode():
    torch.cuda.set_device(0)
    X = synth.power_law(20000, 128, 1.0, device="cuda")
    m = P.saq_fit(X, avg_bits=4.0)
    codes, factors = m.alloc_outputs(X.shape[0])
    m.encode(X, codes, factors)
    torch.cuda.synchronize()
    P.saq_kernel_timing(True)
    l0 = P.saq_kernel_launch_count()
    m.encode(X, codes, factors)
    torch.cuda.synchronize()
    launched = P.saq_kernel_launch_count() - l0
    t = P.saq_kernel_times()
    P.saq_kernel_timing(False)
    ms_p, n_p = t["projection"]
    ms_q, n_q = t["quantize_adjust_pack"]
    ms_o, n_o = t["other"]
    assert n_p >= 1 and n_q >= 1
    assert n_p + n_q + n_o == launched
    assert ms_p > 0 and ms_q > 0
    # nothing more is recorded once timing is off; the record stays readable
    m.encode(X, codes, factors)
    torch.cuda.synchronize()
    assert P.saq_kernel_times() == t
    # starting again clears it
    P.saq_kernel_timing(True)
    assert all(v == (0.0, 0) for v in P.saq_kernel_times().values())
    P.saq_kernel_timing(False)


def test_step_ceiling_measures_and_checks_its_arguments():
    """saq_quantize_step_ceiling: the adjustment step on register-resident
    data at 4 .. 64 resident warps per SM; more warps never cost much."""
    torch.cuda.set_device(0)
    r4 = P.saq_quantize_step_ceiling(4, 4)
    r8 = P.saq_quantize_step_ceiling(8, 4)
    r32 = P.saq_quantize_step_ceiling(32, 4)
    assert r4 > 0 and r8 > 0.9 * r4 and r32 > 0.9 * r8
    for bad in (0, 6, 68):
        with pytest.raises(P.SaqError):
            P.saq_quantize_step_ceiling(bad, 4)
