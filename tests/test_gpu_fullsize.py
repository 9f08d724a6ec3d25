"""Parity at the benchmark sizes, in the launch configuration bench.py times.

The FP64 oracle cannot propagate these grids for thousands of steps in a
test, so it checks what it can compute exactly: the first K samples.  In K
steps the 25-point star stencil moves information at most 4 cells per axis
per step, so for samples n < K the seismograms of the full grid equal those
of the oracle run on a window (aperture) around the source that is wider
than the light cone: the window's own sponge and boundary lie where the
field is still zero.  Everything else is checked through properties that
hold at any size: bitwise identity across work decompositions, storage
modes and batching, and descent of the misfit along the negative gradient.
"""
import dataclasses

import numpy as np
import pytest

from paper_2502_12350_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEIS_TOL_64 = 1e-4
K = 48  # oracle samples (light-cone window half-width 4 K + 8 cells)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2502_12350_gb300 import build, mamute
    build.build()
    c = mamute.Context(0)
    yield c
    c.close()


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)


def run_model(ctx, w, **opts):
    """Device seismograms [n_rec][nt] of the workload (the bench call)."""
    from paper_2502_12350_gb300 import mamute
    dev = torch.device("cuda:0")
    vel = torch.from_numpy(np.ascontiguousarray(w.vel)).to(dev)
    rho = None if w.rho is None else torch.from_numpy(np.ascontiguousarray(w.rho)).to(dev)
    seis = torch.full((int(w.rec_offset[-1]), w.nt), float("nan"), device=dev)
    ctx.model(mamute.grid_of(w), vel, rho, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, seis,
              aperture=w.aperture, **opts)
    return seis


def light_cone_window(w, shot, rec_lo, rec_hi):
    """Aperture (x0, x1, y0, y1) of half-width 4 K + 8 around the shot's
    source (x0 on a multiple of 4) and the shot's receivers inside it."""
    sx, sy = (int(round(c / w.h)) for c in w.src_xyz[shot][:2])
    r = 4 * K + 8
    x0 = max(0, sx - r)
    x0 -= x0 % 4
    x1, y0, y1 = min(w.nx, sx + r), max(0, sy - r), min(w.ny, sy + r)
    ix = np.rint(w.rec_xyz[rec_lo:rec_hi, 0] / w.h).astype(int)
    iy = np.rint(w.rec_xyz[rec_lo:rec_hi, 1] / w.h).astype(int)
    inside = np.nonzero((ix >= x0) & (ix < x1) & (iy >= y0) & (iy < y1))[0] + rec_lo
    return (x0, x1, y0, y1), inside


def oracle_first_samples(oracle, w, shot, aperture, recs):
    og = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, K)
    return oracle.model(og, w.vel, w.src_xyz[shot:shot + 1], w.wavelet[:K],
                        np.array([0, len(recs)], np.int32), w.rec_xyz[recs], rho=w.rho,
                        aperture=np.array([aperture], np.int32))


@pytest.fixture(scope="module")
def headline(ctx):
    w = synth.forward_density()  # 512x512x256 with density, 4000 steps
    return w, run_model(ctx, w)


def test_headline_model_first_samples_match_oracle(headline, oracle):
    w, seis = headline
    assert bool(torch.isfinite(seis).all())
    ap, recs = light_cone_window(w, 0, 0, int(w.rec_offset[1]))
    assert len(recs) > 1000
    got = seis[torch.from_numpy(recs).to(seis.device), :K].cpu().numpy()
    ref = oracle_first_samples(oracle, w, 0, ap, recs)
    assert np.abs(ref).max() > 0
    assert rel(got, ref) <= SEIS_TOL_64


def test_headline_model_bitwise_across_decompositions(ctx, headline):
    """The benchmark's launch configuration (the cost model's tiles), a forced
    64x16 tile in 2 z blocks, and two time steps per launch on the two-level
    kernel give the same bits on the full grid."""
    w, seis = headline
    other = run_model(ctx, w, tiles=[64, 16, 2, 0, 0, 0])
    assert bool(torch.equal(seis, other))
    two = run_model(ctx, w, time_blocking=2)
    assert bool(torch.equal(seis, two))


def test_gradient_256cube_storage_modes_and_descent(ctx):
    """The 256^3 single-shot gradient: automatic storage (every imaging term
    kept, the benchmark's configuration) equals 16-slot binomial
    checkpointing bit for bit, and a small step along -grad lowers the
    misfit by the amount the gradient predicts."""
    from paper_2502_12350_gb300 import mamute
    w = synth.gradient_single()
    dev = torch.device("cuda:0")
    dobs = run_model(ctx, w)
    wi = dataclasses.replace(w, vel=w.vel_init)
    g = mamute.grid_of(wi)
    v0 = torch.from_numpy(np.ascontiguousarray(wi.vel)).to(dev)
    grads = []
    for ns in (0, 16):
        grad = torch.full_like(v0, float("nan"))
        J = ctx.gradient(g, v0, None, wi.src_xyz, wi.wavelet, wi.rec_offset, wi.rec_xyz, dobs,
                         grad, n_snapshots=ns)
        grads.append((J, grad))
    (J0, g0), (J1, g1) = grads
    assert J0 == J1 and J0 > 0
    assert bool(torch.equal(g0, g1))
    assert bool(torch.isfinite(g0).all()) and float(g0.abs().max()) > 0
    # First-order check along -grad, away from the acquisition layer and the
    # outer model layer (whose edge replication into the sponge the gradient
    # leaves out): J(c + eps d) - J(c) ~ eps <grad, d> for a 0.5 m/s step.
    gn = g0.cpu().numpy().astype(np.float64)
    d = np.zeros_like(gn)
    d[16:-1, 1:-1, 1:-1] = -gn[16:-1, 1:-1, 1:-1]
    eps = 0.5 / np.abs(d).max()
    pred = eps * float(np.sum(gn * d))
    seis = run_model(ctx, dataclasses.replace(wi, vel=(wi.vel + eps * d).astype(np.float32)))
    dJ = 0.5 * float(((seis.double() - dobs.double()) ** 2).sum()) - J0
    assert dJ < 0 and 0.5 < dJ / pred < 1.5, (dJ, pred)


def test_batched_shots_match_single_shots_and_oracle(ctx, oracle):
    """64 shots with their own apertures in one launch per step (the
    benchmark's configuration): two shots equal their single-shot runs bit
    for bit, and the first samples of one equal the oracle's."""
    w = synth.batched_shots()
    seis = run_model(ctx, w)
    assert bool(torch.isfinite(seis).all())
    for s in (0, 37):
        lo, hi = int(w.rec_offset[s]), int(w.rec_offset[s + 1])
        one = dataclasses.replace(w, src_xyz=w.src_xyz[s:s + 1],
                                  rec_offset=np.array([0, hi - lo], np.int32),
                                  rec_xyz=w.rec_xyz[lo:hi], aperture=w.aperture[s:s + 1])
        assert bool(torch.equal(run_model(ctx, one), seis[lo:hi]))
    s = 37
    lo, hi = int(w.rec_offset[s]), int(w.rec_offset[s + 1])
    ap, recs = light_cone_window(w, s, lo, hi)
    x0, x1, y0, y1 = w.aperture[s]
    ap = (max(ap[0], x0), min(ap[1], x1), max(ap[2], y0), min(ap[3], y1))  # within the shot's own window
    assert ap[0] % 4 == 0
    got = seis[torch.from_numpy(recs).to(seis.device), :K].cpu().numpy()
    ref = oracle_first_samples(oracle, w, s, ap, recs)
    assert np.abs(ref).max() > 0
    assert rel(got, ref) <= SEIS_TOL_64
