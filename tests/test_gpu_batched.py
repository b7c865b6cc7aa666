"""GPU batched forward: each image of one plan runs the variant the tuning
table names for its (kind, radius bucket, order bucket) (or the built-in
choice) and equals the single-image call with that variant bit for bit;
graph replays are identical; sampled pixels match the checker."""
import contextlib

import numpy as np
import pytest
import torch

import oracle
import paper_1603_08109_gb300 as bf
from helpers import compare_forward, image, needs_gpu, scaled_q, spatial
from paper_1603_08109_gb300 import synth

pytestmark = [pytest.mark.gpu, needs_gpu]


def _batch(specs):
    imgs, outs, host = [], [], []
    for sp in specs:
        a = image(sp["height"], sp["width"], seed=sp["seed"])
        host.append(a)
        imgs.append(torch.from_numpy(a).cuda())
        outs.append(torch.empty_like(imgs[-1]))
    return host, imgs, outs


def _with_order(specs):
    for sp in specs:
        sp["N"] = bf.order_from_delta(sp["kind"], sp["radius"], sp["sigma_s"], sp["sigma_r"], 1.0)
    return specs


def _single(img, sp, variant):
    return bf.gpa_forward(img, sp["kind"], sp["sigma_r"], sp["N"], radius=sp["radius"],
                          sigma_s=sp["sigma_s"], variant=variant)


def _key(sp):
    return sp["kind"], bf.radius_bucket(sp["radius"]), bf.order_bucket(sp["N"])


@contextlib.contextmanager
def _table(entries):
    """Set tuning-table entries {(kind, rb, ob): variant} (and clear every
    other entry of those kinds) for the duration of a block."""
    saved = {}
    for kind in (bf.BOX, bf.GAUSS):
        for rb in range(8):
            for ob in range(6):
                saved[(kind, rb, ob)] = bf.tuning_get(kind, rb, ob)
                bf.tuning_set(kind, rb, ob, entries.get((kind, rb, ob), -1))
    try:
        yield
    finally:
        for k, v in saved.items():
            bf.tuning_set(*k, v)


def _check_plan(specs, host, imgs, outs, where):
    plan = bf.BatchPlan(imgs, outs, specs)
    variants = plan.variants()
    items, ctas = plan.info()
    assert items >= len(specs) and ctas >= 0
    plan.run()
    torch.cuda.synchronize()
    assert int(plan.status.item()) == 0
    first = [o.clone() for o in outs]
    for x, o, sp, v in zip(imgs, first, specs, variants):
        assert torch.equal(o, _single(x, sp, v)), (where, sp, v)
    for _ in range(3):
        for o in outs:
            o.fill_(-1.0)
        plan.replay()
        torch.cuda.synchronize()
        for o, f in zip(outs, first):
            assert torch.equal(o, f)
    plan.close()
    return variants, first


def test_batched_equals_single_image_kernel_and_graph_replays():
    """Built-in choices (empty table): compile-time-radius, runtime-radius and
    banded images in one plan, a 1 x 1 image, a thin image at a large radius."""
    specs = _with_order(synth.batch_specs(12, seed=77, max_hw=(300, 400)))
    specs[0].update(radius=45, sigma_s=15.0, kind=bf.GAUSS)
    specs[1].update(height=1, width=1)
    specs[2].update(height=3, width=700, kind=bf.BOX, radius=30)
    specs[3].update(radius=9, sigma_s=3.0, kind=bf.GAUSS)
    specs[4].update(radius=7, sigma_s=7 / 3.0, kind=bf.BOX)
    _with_order(specs)
    host, imgs, outs = _batch(specs)
    with _table({}):
        variants, first = _check_plan(specs, host, imgs, outs, "built-in")
    assert variants[0] == bf.BANDED_VARIANT and variants[2] == bf.BANDED_VARIANT
    assert variants[3] == 5 and variants[4] in range(5)
    for k in (0, 3, 4):
        sp = specs[k]
        w = spatial(sp["kind"], sp["radius"], sp["sigma_s"])
        ro, P, Q = oracle.gpa_alg2(host[k], w, sp["sigma_r"], sp["N"], return_parts=True)
        compare_forward(first[k].cpu().numpy(), None, ro, scaled_q(host[k], Q, sp["sigma_r"]),
                        w[sp["radius"], sp["radius"]], "batched %d" % k, sigma_r=sp["sigma_r"],
                        N=sp["N"], img=host[k], w=w)


def test_batched_follows_the_tuning_table():
    """Table entries drive each image's variant: every runtime-radius tile
    shape (one persistent launch each), the banded forward at a small radius,
    the compile-time-radius kernel; an entry that does not fit the image's
    radius (variant 5 at W = 7) falls back to the built-in choice."""
    base = [(bf.GAUSS, 4, 4 / 3.0, 40.0), (bf.GAUSS, 6, 2.0, 30.0), (bf.BOX, 10, 0.0, 50.0),
            (bf.GAUSS, 9, 3.0, 60.0), (bf.BOX, 7, 0.0, 35.0), (bf.GAUSS, 14, 14 / 3.0, 70.0),
            (bf.BOX, 22, 0.0, 25.0), (bf.GAUSS, 25, 25 / 3.0, 45.0)]
    specs = []
    for k, (kind, r, ss, sr) in enumerate(base):
        for j in range(2):
            specs.append({"height": 90 + 37 * k + 11 * j, "width": 130 + 53 * k + 7 * j,
                          "kind": kind, "radius": r, "sigma_s": ss, "sigma_r": sr,
                          "seed": 900 + 10 * k + j})
    _with_order(specs)
    host, imgs, outs = _batch(specs)
    want = {0: 1, 1: 3, 2: 4, 3: 5, 4: 5, 5: 2, 6: 0, 7: bf.BANDED_VARIANT}
    entries = {_key(specs[2 * k]): v for k, v in want.items()}
    assert len(entries) == len(want)  # the cases sit in distinct buckets
    with _table(entries):
        variants, first = _check_plan(specs, host, imgs, outs, "tuned")
    for k, v in want.items():
        exp = v if not (v == 5 and specs[2 * k]["radius"] not in (3, 5, 9, 15)) else None
        for j in range(2):
            got = variants[2 * k + j]
            if exp is None:
                assert got != 5 and got in range(5), (k, got)
            else:
                assert got == exp, (k, j, got, exp)
    rng = np.random.default_rng(5)
    for k in range(0, len(specs), 3):
        sp = specs[k]
        ys = rng.integers(0, sp["height"], 30)
        xs = rng.integers(0, sp["width"], 30)
        w = spatial(sp["kind"], sp["radius"], sp["sigma_s"])
        ro, P, Q = oracle.gpa_alg2_at(host[k], w, sp["sigma_r"], sp["N"], (ys, xs),
                                      return_parts=True)
        compare_forward(first[k].cpu().numpy()[ys, xs], None, ro,
                        scaled_q(host[k][ys, xs], Q, sp["sigma_r"]), w[sp["radius"], sp["radius"]],
                        "tuned batch %d" % k, sigma_r=sp["sigma_r"], N=sp["N"], img=host[k], w=w,
                        pixels=(ys, xs))


def test_banded_variant_at_small_radii_matches_checker():
    """The banded forward chosen explicitly at radii the built-in rule gives
    to the fused kernels (both kinds), against the checker."""
    img = image(150, 290, seed=44)
    for kind, r, ss, sr, N in ((bf.GAUSS, 3, 1.0, 40.0, 12), (bf.BOX, 5, 0.0, 30.0, 41),
                               (bf.GAUSS, 9, 3.0, 30.0, 40), (bf.BOX, 1, 0.0, 60.0, 2)):
        out, q = bf.gpa_forward(torch.from_numpy(img).cuda(), kind, sr, N, radius=r, sigma_s=ss,
                                return_q=True, variant=bf.BANDED_VARIANT)
        w = spatial(kind, r, ss)
        ro, P, Q = oracle.gpa_alg2(img, w, sr, N, return_parts=True)
        compare_forward(out.cpu().numpy(), q.cpu().numpy(), ro, scaled_q(img, Q, sr), w[r, r],
                        "banded kind %d r %d N %d" % (kind, r, N), sigma_r=sr, N=N, img=img, w=w)


def test_batched_full_256_workload():
    """The uneven 256-image batch: every image equals the single-image call
    with the variant the plan chose for it."""
    specs = _with_order(synth.batch_specs(256, seed=3000))
    host, imgs, outs = _batch(specs)
    with _table({}):
        plan = bf.BatchPlan(imgs, outs, specs)
        variants = plan.variants()
        plan.replay()
        torch.cuda.synchronize()
    for x, o, sp, v in zip(imgs, outs, specs, variants):
        assert torch.equal(o, _single(x, sp, v))
    k = int(np.argmax([sp["N"] for sp in specs]))
    sp = specs[k]
    rng = np.random.default_rng(1)
    ys = rng.integers(0, sp["height"], 40)
    xs = rng.integers(0, sp["width"], 40)
    w = spatial(sp["kind"], sp["radius"], sp["sigma_s"])
    ro, P, Q = oracle.gpa_alg2_at(host[k], w, sp["sigma_r"], sp["N"], (ys, xs), return_parts=True)
    compare_forward(outs[k].cpu().numpy()[ys, xs], None, ro,
                    scaled_q(host[k][ys, xs], Q, sp["sigma_r"]), w[sp["radius"], sp["radius"]],
                    "batched max-N image", sigma_r=sp["sigma_r"], N=sp["N"], img=host[k], w=w,
                    pixels=(ys, xs))
    plan.close()
