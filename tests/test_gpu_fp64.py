"""The step kernels replace IEEE division and sqrt by a hardware seed plus one
third-order series step; check those against CUDA's correctly rounded results."""
import ctypes as C

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_fast_rcp_and_sqrt_within_a_few_ulp():
    from paper_2107_06355_gb300 import _lib as L

    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = L.lib().pplbm_fp64_selftest(1 << 24, 12345, C.c_void_p(out.data_ptr()),
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    err_rcp, err_sqrt = out.tolist()
    ulp = 2.0**-52
    assert err_rcp <= 2 * ulp, err_rcp
    assert err_sqrt <= 2 * ulp, err_sqrt


def test_fp64_peak_probe_reports_a_rate_consistent_with_its_own_timing():
    """pplbm_fp64_peak (the denominator of the step's FP64 roofline): the rate equals
    the instructions it issues over the launch time it reports, and stays within the
    nominal issue rate of the part (2 FP64 FMA per clock per SM at the maximum clock)
    with some margin for clock reporting."""
    from paper_2107_06355_gb300 import _lib as L

    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = (C.c_double * 3)()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for chains, op in ((8, 0), (1, 0), (32, 0), (8, 1), (8, 2)):
        assert L.lib().pplbm_fp64_peak(4, chains, op, 20000, C.c_void_p(sink.data_ptr()), out, stream) == 0
        rate, ms, blocks = out[0], out[1], int(out[2])
        assert blocks == 4 * sms
        assert rate == pytest.approx(blocks * 256 * 20000 * chains / (ms * 1e-3), rel=1e-12)
        assert 0.05e12 < rate < 1.2 * 2 * sms * 2.1e9
    assert sink.item() == 0.0
    # the integer-pipe additions run beside the FP64 FMAs: both together take no longer
    # than the slower of the two alone (within 10 %)
    t = {}
    for op in (0, 3, 4):
        assert L.lib().pplbm_fp64_peak(8, 8, op, 20000, C.c_void_p(sink.data_ptr()), out, stream) == 0
        t[op] = out[1]
    assert t[4] < 1.1 * max(t[0], t[3])
    for bad in ((0, 8, 0, 10), (65, 8, 0, 10), (4, 8, 0, 0), (4, 3, 0, 10), (4, 8, 7, 10), (4, 8, -1, 10)):
        assert L.lib().pplbm_fp64_peak(*bad, C.c_void_p(sink.data_ptr()), out, stream) == L.PPLBM_ERR_ARG


def test_integer_pipe_addition_is_bitwise_the_fp64_add():
    """add_pos_int (the density pass's sums of positive populations on the integer
    pipe) against the FP64 pipe's x + y on 2^30 seeded pairs: random exponents,
    exponent gaps 0..63, exact ties and rounding carries; no bit may differ."""
    from paper_2107_06355_gb300 import _lib as L

    out = torch.zeros(5, dtype=torch.int64, device="cuda")
    st = L.lib().pplbm_int_add_selftest(1 << 30, 20260, C.c_void_p(out.data_ptr()),
                                        C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    bad = out.tolist()
    assert bad[0] == 0, [hex(v & (2**64 - 1)) for v in bad]


def test_fixed_point_sums_device_build_equals_host_build(fixsum_host):
    """The step kernels' fixed-point moments and stencil sums (fixsum.cuh) compiled for
    sm_103a give bit for bit the results of the host build of the same source, which
    test_fixsum_host.py checks against exact rational sums: 2^20 population sets
    (interface-like and independent exponents, a few outside the range) and psi
    stencils (smooth, across interfaces, with non-finite and negative entries)."""
    import numpy as np

    from paper_2107_06355_gb300 import _lib as L

    rng = np.random.default_rng(2107)
    n = 1 << 20
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    f = w * 10.0 ** rng.uniform(-6, 0, size=(n, 1)) * (1 + rng.uniform(-0.99, 0.99, size=(n, 9)))
    k = n // 4
    f[:k] = np.ldexp(1 + rng.random((k, 9)), rng.integers(-70, 30, size=(k, 9)))
    f[k:k + 64, 3] = [0.0, -1e-3, np.inf, np.nan] * 16
    p = 10.0 ** rng.uniform(-3, 1, size=(n, 1)) * (1e-3 + rng.random((n, 8)))
    p[:1000, 2] = [np.inf, np.nan, -0.5, 0.0] * 250
    host_d = np.zeros((n, 6))
    host_s = np.zeros((n, 2))
    fixsum_host.fx_density(n, f.ctypes.data, host_d.ctypes.data)
    fixsum_host.fx_stencil(n, p.ctypes.data, host_s.ctypes.data)
    fd, pd = torch.from_numpy(f).cuda(), torch.from_numpy(p).cuda()
    out = torch.empty((n, 8), dtype=torch.float64, device="cuda")
    st = L.lib().pplbm_fixsum_eval(n, C.c_void_p(fd.data_ptr()), C.c_void_p(pd.data_ptr()),
                                   C.c_void_p(out.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    dev = out.cpu().numpy()
    # bit patterns (NaN payloads included)
    assert np.array_equal(dev[:, :6].view(np.int64), host_d.view(np.int64))
    assert np.array_equal(dev[:, 6:].view(np.int64), host_s.view(np.int64))
    assert dev[:, 5].sum() < n and dev[:, 5].sum() > n - 100
    assert L.lib().pplbm_fixsum_eval(-1, None, None, None, None) == L.PPLBM_ERR_ARG
    assert L.lib().pplbm_fixsum_eval(4, None, None, None, None) == L.PPLBM_ERR_ARG
    assert L.lib().pplbm_fixsum_eval(0, None, None, None, None) == 0


@pytest.mark.parametrize("shear", [0, 1])
def test_collision_fixed_point_device_build_equals_host_build(fixsum_host, shear):
    """The collision pass's fixed-point output stage and j/h sums (fixsum.cuh) compiled
    for sm_103a against the host build of the same source (checked in
    test_fixsum_host.py against the populations' definition): bit for bit on 2^20 rows
    in the bulk, interface and Li-dominated regimes, with zeros and non-finite inputs."""
    import numpy as np

    from paper_2107_06355_gb300 import _lib as L

    rng = np.random.default_rng(36 + shear)
    n = 1 << 20
    rho = 10.0 ** rng.uniform(-5, 0, size=n)
    scale = np.choose(rng.integers(0, 3, size=n), [1e-4, 0.3, 1.0])
    q = rng.normal(size=(n, 9)) * (rho * scale / 36)[:, None]
    q[:, 0] = rho / 36
    q[::3, 6] = rho[::3] * 10.0 ** rng.uniform(1, 4, size=q[::3].shape[0])
    q[:1000, 1:] = 0.0
    q[1000:1010, 5] = np.inf
    q[1010:1020, 7] = np.nan
    jh = rng.normal(size=(n, 2)) * 10.0 ** rng.uniform(-8, 0, size=(n, 2))
    jh[:500, 0] = 0.0
    jh[500:1000, 1] = -0.0
    host = np.zeros((n, 9))
    sh = np.ascontiguousarray(q)
    fixsum_host.fx_populations(n, shear, sh.ctypes.data, host.ctypes.data)
    hj = np.zeros((n, 4))
    fixsum_host.fx_j_h(n, jh.ctypes.data, hj.ctypes.data)
    qd, jd = torch.from_numpy(q).cuda(), torch.from_numpy(jh).cuda()
    out = torch.empty((n, 13), dtype=torch.float64, device="cuda")
    st = L.lib().pplbm_fixsum_collision_eval(n, shear, C.c_void_p(qd.data_ptr()), C.c_void_p(jd.data_ptr()),
                                             C.c_void_p(out.data_ptr()),
                                             C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    dev = out.cpu().numpy()
    assert np.array_equal(dev[:, :9].view(np.int64), host.view(np.int64))
    assert np.array_equal(dev[:, 9:].view(np.int64), hj.view(np.int64))
    assert L.lib().pplbm_fixsum_collision_eval(-1, 0, None, None, None, None) == L.PPLBM_ERR_ARG
    assert L.lib().pplbm_fixsum_collision_eval(2, 0, None, None, None, None) == L.PPLBM_ERR_ARG


@pytest.mark.parametrize("shear", [0, 1])
def test_adjoint_fixed_point_device_build_equals_host_build(fixsum_host, shear):
    """The adjoint's fixed-point stages (fixsum.cuh: the transposed output stage and
    sums of the collision pass, the psi gather and lambda assembly of the density pass)
    compiled for sm_103a against the host build (checked in test_fixsum_host.py against
    derivatives of the populations' definition, the stencil's transpose and the moment
    rows): bit for bit on 2^20 rows, with zeros and non-finite inputs."""
    import numpy as np

    from paper_2107_06355_gb300 import _lib as L

    rng = np.random.default_rng(90 + shear)
    n = 1 << 20
    mu = rng.normal(size=(n, 9)) * 10.0 ** rng.uniform(-6, 2, size=(n, 1))
    mu[:5000] *= 10.0 ** rng.uniform(-3, 0, size=(5000, 9))
    mu[5000:5100, 2] = 0.0
    mu[5100:5110, 7] = np.nan
    a = rng.normal(size=(n, 6)) * 10.0 ** rng.uniform(-8, 1, size=(n, 6))
    a[:300, 3] = 0.0
    a[300:310, 5] = np.inf
    gth = rng.normal(size=(n, 13)) * 10.0 ** rng.uniform(-6, 1, size=(n, 13))
    gth[:200, 0] = 0.0
    gth[200:210, 7] = np.nan
    lam = rng.normal(size=(n, 5)) * 10.0 ** rng.uniform(-6, 1, size=(n, 5))
    lam[:100, 3:] = 0.0
    host_u = np.zeros((n, 9))
    host_j = np.zeros((n, 2))
    host_g = np.zeros(n)
    host_l = np.zeros((n, 9))
    fixsum_host.fx_populations_transpose(n, shear, np.ascontiguousarray(mu).ctypes.data, host_u.ctypes.data)
    fixsum_host.fx_j_h_transpose(n, np.ascontiguousarray(a).ctypes.data, host_j.ctypes.data)
    fixsum_host.fx_psi_gather(n, np.ascontiguousarray(gth).ctypes.data, host_g.ctypes.data)
    fixsum_host.fx_lambda(n, shear, np.ascontiguousarray(lam).ctypes.data, host_l.ctypes.data)
    dev_in = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (mu, a, gth, lam)]
    out = torch.empty((n, 21), dtype=torch.float64, device="cuda")
    st = L.lib().pplbm_fixsum_adjoint_eval(n, shear, *[C.c_void_p(t.data_ptr()) for t in dev_in],
                                           C.c_void_p(out.data_ptr()),
                                           C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    dev = out.cpu().numpy()
    assert np.array_equal(dev[:, :9].view(np.int64), host_u.view(np.int64))
    assert np.array_equal(dev[:, 9:11].view(np.int64), host_j.view(np.int64))
    assert np.array_equal(dev[:, 11].view(np.int64), host_g.view(np.int64))
    assert np.array_equal(dev[:, 12:].view(np.int64), host_l.view(np.int64))
    assert L.lib().pplbm_fixsum_adjoint_eval(-1, 0, None, None, None, None, None, None) == L.PPLBM_ERR_ARG
