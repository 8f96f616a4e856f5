"""The allocation-free equation-scale entry point (for callers that cannot
allocate device memory) against the solver's own scales.

Runs last (file name) so that a failure here leaves every other test run.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_scales_match_solver_scales_twice():
    torch = pytest.importorskip("torch")
    from paper_1902_00095_gb300 import thermo
    from synthetic import make_problem
    from synthetic.recipes import perturbed_state
    import ctypes as C

    lib = thermo.load()
    dev = torch.device("cuda:0")
    results = []
    for shape, seed in (((13, 11, 7), 3), ((40, 33, 9), 4)):
        prob = make_problem("tiny", shape=shape, seed=seed)
        p, T = perturbed_state(prob, seed=seed)
        s = thermo.Solver.from_problem(prob)
        s.assemble(p, T, prob["p_n"], prob["T_n"], prob["dt"])
        rp, col, val, sv, scales = s.export_system()
        d_rp = torch.as_tensor(rp, dtype=torch.int32, device=dev)
        d_col = torch.as_tensor(col, dtype=torch.int32, device=dev)
        d_val = torch.as_tensor(val.reshape(-1), dtype=torch.float64, device=dev)
        for call in range(2):
            out = torch.full((2,), -1.0, dtype=torch.float64, device=dev)
            st = lib.tp_equation_scales_noalloc(
                s.N, C.c_void_p(d_rp.data_ptr()), C.c_void_p(d_col.data_ptr()),
                C.c_void_p(d_val.data_ptr()), C.c_void_p(out.data_ptr()), None)
            assert st == thermo.TP_OK
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.all(np.abs(got / scales - 1.0) <= 1e-13), (call, got, scales)
            results.append(got)
        s.close()
    # the two calls on the same input agree exactly (the shared scratch keeps
    # no state between calls)
    assert np.array_equal(results[0], results[1]) and np.array_equal(results[2], results[3])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1902_00095_gb300 import thermo
    import ctypes as C
    lib = thermo.load()
    dummy = C.c_void_p(1)
    assert lib.tp_equation_scales_noalloc(8388609, dummy, dummy, dummy, dummy, None) == thermo.TP_EINVAL
    assert lib.tp_equation_scales_noalloc(0, dummy, dummy, dummy, dummy, None) == thermo.TP_EINVAL
