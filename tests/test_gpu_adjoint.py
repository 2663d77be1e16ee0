"""Differentiable post-path (frozen visibility): forward against the FP64
oracle, the colour gradient against the forward map (adjoint identity), the
lens gradient against central finite differences (h = 1e-3) of the GPU and of
the oracle, and a 200-step Adam fit of focus and aperture."""
import numpy as np
import pytest

import hdof_inputs as hi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2210_04981_gb300.hdof as H  # noqa: E402
from gpu_util import bvh_of, frac_close, host, report  # noqa: E402


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle
    oracle.build()
    return oracle


def _setup(W, Hh, seed=0, with_history=True):
    """Colour/depth of the differentiable workload, a 100k-triangle room
    traced at the target lens (frozen visibility) and frozen history."""
    col, z = hi.diff_inputs(W, Hh, seed)
    scene = hi.room_scene_target(seed, 100_000, aspect=W / Hh)
    cam = hi.Camera(width=W, height=Hh).f32()
    target = hi.Lens(2.5, 0.04, 0.05).f32()
    p = hi.room_params(r_max=32.0, camera_moved=0)
    # mask of the room frame (its own G-buffer) decides which pixels are traced
    bvh = bvh_of(scene)
    r = H.Renderer(bvh, W, Hh, p)
    H.hdof_gbuffer(bvh, cam, cam, p, r.g)
    H.hdof_mask(r.g, None, p, r.edge, r.spp, r.ws)
    H.hdof_sync()
    spp = r.spp.clone()
    n_rays = int(spp.to(torch.int64).sum())
    rec = torch.empty((max(n_rays, 1), 4), dtype=torch.float32, device="cuda")
    ray_off = torch.empty((Hh, W), dtype=torch.int32, device="cuda")
    H.hdof_trace(bvh, cam, target, p, spp, r.rt, r.stats, r.ws, rec=rec, ray_off=ray_off)
    H.hdof_sync()
    hs = hi.random_hist_samples(W, Hh, seed) if with_history else None
    return dict(col=col, z=z, scene=scene, cam=cam, target=target, p=p, spp=spp, rec=rec, ray_off=ray_off, hs=hs)


def _oracle_side(orc, s):
    """The oracle's own mask and hit records for the same room frame."""
    osc = orc.OScene(s["scene"])
    g = orc.gbuffer(osc, s["cam"], s["cam"], s["p"])
    spp = orc.mask(g["nd"], g["mv"], s["p"])["spp"]
    rec, off = orc.trace_records(osc, s["cam"], s["target"], s["p"], spp)
    return spp, rec, off


def _path(s):
    zt = torch.from_numpy(s["z"]).cuda()
    hs = torch.from_numpy(s["hs"]).cuda() if s["hs"] is not None else None
    return H.PostPath(zt, s["spp"], s["rec"], s["ray_off"], hs, s["cam"], s["p"])


def test_post_forward_matches_oracle(orc):
    W, Hh = 160, 120
    s = _setup(W, Hh)
    path = _path(s)
    out = host(path.forward(torch.from_numpy(s["col"]).cuda(), 2.0, 0.03))
    spp, rec, off = _oracle_side(orc, s)
    assert (spp == host(s["spp"])).mean() >= 0.999
    ref = orc.post_forward(s["col"].astype(np.float64), s["z"].astype(np.float64), spp, rec, off,
                           s["hs"].astype(np.float64), s["cam"], hi.Lens(2.0, 0.03, 0.05).f32(), s["p"])
    assert (spp > 0).mean() > 0.05
    tr = spp > 0
    assert frac_close(host(path.st.crt)[tr], ref["crt"][tr], 1e-3, 1e-3) >= 0.999
    assert frac_close(out, ref["out"][..., :3], 1e-3) >= 0.999, report("out", out, ref["out"][..., :3])


def test_colour_gradient_is_the_adjoint(orc):
    """out is linear in the colour image: <J x, y> = <x, J^T y>."""
    W, Hh = 192, 128
    s = _setup(W, Hh, seed=1)
    path = _path(s)
    zf, A = 2.2, 0.035
    C = torch.from_numpy(s["col"]).cuda()
    rng = np.random.default_rng(2)
    x = torch.from_numpy(rng.normal(size=(Hh, W, 3)).astype(np.float32)).cuda()
    y = torch.from_numpy(rng.normal(size=(Hh, W, 3)).astype(np.float32)).cuda()
    o0 = path.forward(C, zf, A).double().clone()
    o1 = path.forward(C + x, zf, A).double().clone()
    Jx = o1 - o0
    path.forward(C, zf, A)
    gcol, _ = path.backward(y, zf, A)
    lhs = float((Jx * y.double()).sum())
    rhs = float((x.double() * gcol.double()).sum())
    assert abs(lhs - rhs) <= 1e-4 * max(abs(lhs), 1e-6), (lhs, rhs)
    # the oracle's forward map gives the same J x (FP64, linear in C)
    spp, rec, off = _oracle_side(orc, s)
    lens = hi.Lens(zf, A, 0.05)
    hs = s["hs"].astype(np.float64)
    r0 = orc.post_forward(s["col"].astype(np.float64), s["z"].astype(np.float64), spp, rec, off, hs, s["cam"],
                          lens, s["p"])["out"][..., :3]
    r1 = orc.post_forward(s["col"].astype(np.float64) + host(x), s["z"].astype(np.float64), spp, rec, off, hs,
                          s["cam"], lens, s["p"])["out"][..., :3]
    ref = float(((r1 - r0) * host(y)).sum())
    assert abs(ref - rhs) <= 1e-3 * abs(ref), (ref, rhs)


def test_colour_gradient_equals_the_oracle_vjp(orc):
    """grad_col element by element against the oracle's J^T g (its Jacobian
    in the colour image by definition, FP64: oracle.post_colour_vjp).  Both
    sides take the same seeded mask (left half untraced, 1-8 rays elsewhere)
    and trace their own hit records of the same room at the target lens."""
    W, Hh = 32, 24
    col, z = hi.diff_inputs(W, Hh, 3)
    scene = hi.room_scene_target(3, 100_000, aspect=W / Hh)
    cam = hi.Camera(width=W, height=Hh).f32()
    target = hi.Lens(2.5, 0.04, 0.05).f32()
    p = hi.room_params(r_max=32.0, camera_moved=0)
    rng = np.random.default_rng(11)
    spp = rng.integers(1, 9, (Hh, W)).astype(np.uint8)
    spp[:, : W // 2] = 0
    hs = hi.random_hist_samples(W, Hh, 3)
    g = rng.normal(size=(Hh, W, 3))
    zf, A = 2.2, 0.035
    # GPU: the mask's hit records, then forward and adjoint
    bvh = bvh_of(scene)
    r = H.Renderer(bvh, W, Hh, p)
    spp_d = torch.from_numpy(spp).cuda()
    rec = torch.empty((int(spp.astype(np.int64).sum()), 4), dtype=torch.float32, device="cuda")
    ray_off = torch.empty((Hh, W), dtype=torch.int32, device="cuda")
    H.hdof_trace(bvh, cam, target, p, spp_d, r.rt, r.stats, r.ws, rec=rec, ray_off=ray_off)
    H.hdof_sync()
    path = H.PostPath(torch.from_numpy(z).cuda(), spp_d, rec, ray_off, torch.from_numpy(hs).cuda(), cam, p)
    path.forward(torch.from_numpy(col).cuda(), zf, A)
    gcol, _ = path.backward(torch.from_numpy(g.astype(np.float32)).cuda(), zf, A)
    H.hdof_sync()
    gcol = host(gcol)
    # oracle: its own records of the same rays, its Jacobian by definition
    osc = orc.OScene(scene)
    orec, ooff = orc.trace_records(osc, cam, target, p, spp)
    ref = orc.post_colour_vjp(col.astype(np.float64), z.astype(np.float64), spp, orec, ooff,
                              hs.astype(np.float64), cam, hi.Lens(zf, A, 0.05).f32(), p,
                              g.astype(np.float32).astype(np.float64))
    scale = float(np.abs(ref).max())
    ok = np.abs(gcol - ref) <= 1e-4 * scale
    assert ok.mean() >= 0.999, report("grad_col", gcol, ref)
    assert np.abs(ref - g).max() > 1e-2 * scale  # blur: J is not the identity


def _loss_gpu(path, C, Y, zf, A):
    return float((path.forward(C, zf, A).double() * Y.double()).sum())


def test_lens_gradient_against_finite_differences(orc):
    """Analytic d/d(focus, aperture) against central differences (h = 1e-3)
    of the GPU forward on the 1024x1024 workload.  The post-path is piecewise
    linear at pixel scale (every soft step has kinks), so a central difference
    is the mean derivative over [theta - h, theta + h]: it is compared with
    the adjoint averaged over that interval (Simpson, 9 points); the pointwise
    adjoint is reported next to it."""
    W, Hh = 1024, 1024
    s = _setup(W, Hh, seed=0)
    path = _path(s)
    C = torch.from_numpy(s["col"]).cuda()
    Y = torch.from_numpy(np.random.default_rng(3).uniform(-1, 1, (Hh, W, 3)).astype(np.float32)).cuda()
    zf, A = 2.0, 0.03
    hz, hA = 1e-3, 1e-4  # the aperture is ~0.03: 1e-3 would move it by 3%

    def grad(zf_, A_):
        path.forward(C, zf_, A_)
        return host(path.backward(Y, zf_, A_)[1]).astype(np.float64)

    def mean_grad(k, h):
        ts = np.linspace(-h, h, 9)
        w = np.array([1, 4, 2, 4, 2, 4, 2, 4, 1], np.float64) / 24.0
        return sum(wi * grad(zf + t, A)[k] if k == 0 else wi * grad(zf, A + t)[k] for wi, t in zip(w, ts))

    g0 = grad(zf, A)
    fd_zf = (_loss_gpu(path, C, Y, zf + hz, A) - _loss_gpu(path, C, Y, zf - hz, A)) / (2 * hz)
    fd_A = (_loss_gpu(path, C, Y, zf, A + hA) - _loss_gpu(path, C, Y, zf, A - hA)) / (2 * hA)
    m_zf, m_A = mean_grad(0, hz), mean_grad(1, hA)
    print(f"d/dfocus: adjoint {g0[0]:.5g}, interval mean {m_zf:.5g}, central difference {fd_zf:.5g}")
    print(f"d/daperture: adjoint {g0[1]:.5g}, interval mean {m_A:.5g}, central difference {fd_A:.5g}")
    assert abs(m_zf - fd_zf) <= 1e-2 * abs(fd_zf), (m_zf, fd_zf)
    assert abs(m_A - fd_A) <= 1e-2 * abs(fd_A), (m_A, fd_A)
    assert abs(g0[0] - fd_zf) <= 5e-2 * abs(fd_zf) and abs(g0[1] - fd_A) <= 5e-2 * abs(fd_A)


def test_lens_gradient_against_oracle_fd(orc):
    W, Hh = 160, 120
    s = _setup(W, Hh, seed=4)
    path = _path(s)
    C = torch.from_numpy(s["col"]).cuda()
    Yn = np.random.default_rng(5).uniform(-1, 1, (Hh, W, 3))
    zf, A, h = 2.0, 0.03, 1e-3
    path.forward(C, zf, A)
    _, g = path.backward(torch.from_numpy(Yn.astype(np.float32)).cuda(), zf, A)
    g = host(g)
    spp, rec, off = _oracle_side(orc, s)
    hs = s["hs"].astype(np.float64)

    def L(zf_, A_):
        o = orc.post_forward(s["col"].astype(np.float64), s["z"].astype(np.float64), spp, rec, off, hs, s["cam"],
                             hi.Lens(zf_, A_, 0.05), s["p"])["out"][..., :3]
        return float((o * Yn).sum())

    fd_zf = (L(zf + h, A) - L(zf - h, A)) / (2 * h)
    fd_A = (L(zf, A + h * 0.1) - L(zf, A - h * 0.1)) / (2 * h * 0.1)
    assert abs(g[0] - fd_zf) <= 1e-2 * abs(fd_zf), (g[0], fd_zf)
    assert abs(g[1] - fd_A) <= 1e-2 * abs(fd_A), (g[1], fd_A)


def test_adam_fit_recovers_lens():
    """Target rendered at (2.5, 0.04) with the visibility traced there; 200
    Adam steps from (1.0, 0.02) recover it."""
    W, Hh = 1024, 1024
    s = _setup(W, Hh, seed=0)
    path = _path(s)
    C = torch.from_numpy(s["col"]).cuda()
    target = path.forward(C, 2.5, 0.04).clone()
    # fit in (a, b) = (A / 0.04, (A / zf) / 0.016): the CoC A H (1/z - 1/zf) / t
    # is linear in them, which removes the valley of equal blur along
    # A (1/z - 1/zf) = const that traps a fit in (zf, A); L1 image loss
    a_t = torch.tensor(0.02 / 0.04, device="cuda", requires_grad=True)
    b_t = torch.tensor((0.02 / 1.0) / 0.016, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([a_t, b_t], lr=0.1)
    sched = torch.optim.lr_scheduler.ExponentialLR(opt, gamma=0.98)

    def lens():
        return torch.stack([(0.04 * a_t) / (0.016 * b_t), 0.04 * a_t])

    for _ in range(200):
        opt.zero_grad()
        out = H.HdofPost.apply(C, lens(), path)
        loss = (out - target).abs().mean()
        loss.backward()
        opt.step()
        sched.step()
        with torch.no_grad():
            a_t.clamp_(min=0.01)
            b_t.clamp_(min=0.01)
    theta = lens()
    zf, A = (float(v) for v in theta.detach().cpu())
    assert abs(zf - 2.5) < 0.05 and abs(A - 0.04) < 0.002, (zf, A)


def _step_inputs(s, seed=5):
    W, Hh = s["col"].shape[1], s["col"].shape[0]
    C = torch.from_numpy(s["col"]).cuda()
    Y = torch.from_numpy(np.random.default_rng(seed).uniform(-1, 1, (Hh, W, 3)).astype(np.float32)).cuda()
    return C, Y


def test_device_lens_calls_equal_host_lens_calls():
    """hdof_post_forward_dlens / hdof_post_backward_dlens read (focus,
    aperture) on the device and give the host-record calls' state, image and
    gradients bit for bit."""
    s = _setup(160, 120)
    path = _path(s)
    C, Y = _step_inputs(s)
    zf, A = 2.0, 0.03
    lens_dev = torch.tensor([zf, A], dtype=torch.float32, device="cuda")
    sa, sb = path.new_state(), path.new_state()
    names = ("rt", "crt", "hacc", "mom", "hlen", "crec", "sp_aux", "pp", "pp_aux", "out")
    for st in (sa[0], sb[0]):  # some planes are written at traced pixels only
        for n in names:
            getattr(st, n).zero_()
    path.forward(C, zf, A, sa)
    path.forward_dev(C, lens_dev, sb)
    for n in names:
        assert torch.equal(getattr(sa[0], n), getattr(sb[0], n)), n
    ga, la = path.backward(Y, zf, A, sa)
    gb, lb = path.backward_dev(Y, lens_dev, sb)
    H.hdof_sync()
    assert torch.equal(ga, gb)
    assert torch.equal(la, lb), (la, lb)
    # the autograd op takes the device path: same values as the host-record calls
    out = H.HdofPost.apply(C, lens_dev, path)
    assert torch.equal(out, sa[0].out[..., :3])


def test_post_step_captured_in_a_graph():
    """A forward + backward step with the lens on the device, captured into a
    CUDA graph once and replayed after new lens values are written into the
    same array, equals the eager host-record calls at those values."""
    s = _setup(160, 120)
    path = _path(s)
    C, Y = _step_inputs(s)
    lens_dev = torch.tensor([2.0, 0.03], dtype=torch.float32, device="cuda")
    state = path.new_state()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # warm-up outside the capture (the first calls load a table)
        path.forward_dev(C, lens_dev, state)
        path.backward_dev(Y, lens_dev, state)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        out = path.forward_dev(C, lens_dev, state)
        gcol, glens = path.backward_dev(Y, lens_dev, state)
    for zf, A in ((2.7, 0.045), (1.6, 0.02), (2.0, 0.03)):
        lens_dev.copy_(torch.tensor([zf, A], dtype=torch.float32))
        g.replay()
        ref = path.new_state()
        o_ref = path.forward(C, zf, A, ref).clone()
        g_ref, l_ref = path.backward(Y, zf, A, ref)
        H.hdof_sync()
        assert torch.equal(out, o_ref), (zf, A)
        assert torch.equal(gcol, g_ref), (zf, A)
        assert torch.equal(glens, l_ref), (zf, A, glens, l_ref)

