"""Tile-shape tuning table: JSON cache round trip (CPU) and a small on-GPU
autotune whose chosen variant still meets the parity bar."""
import json

import numpy as np
import pytest
import torch

import oracle
import paper_1603_08109_gb300 as bf
from helpers import compare_forward, image, needs_gpu, scaled_q, spatial
from paper_1603_08109_gb300 import tuning


def test_json_cache_roundtrip(tmp_path):
    path = tmp_path / "tune.json"
    rb, ob = bf.radius_bucket(20), bf.order_bucket(100)
    old = bf.tuning_get(0, rb, ob)
    entries = [{"kind": 0, "radius_bucket": rb, "order_bucket": ob, "variant": 2, "ms": 1.0}]
    path.write_text(json.dumps({"device": "test", "entries": entries}))
    try:
        assert tuning.load(str(path)) == 1
        assert bf.tuning_get(0, rb, ob) == 2
    finally:
        bf.tuning_set(0, rb, ob, old)
    assert tuning.load(str(tmp_path / "missing.json")) == 0


@pytest.fixture
def restored_table():
    """The tuning table is process-wide: put back every entry a test changed."""
    saved = {(k, rb, ob): bf.tuning_get(k, rb, ob)
             for k in (bf.BOX, bf.GAUSS) for rb in range(8) for ob in range(6)}
    yield
    for key, v in saved.items():
        bf.tuning_set(*key, v)


@pytest.mark.gpu
@needs_gpu
def test_autotune_then_forward_meets_parity(tmp_path, restored_table):
    entries = tuning.autotune_grid(128, 300, kinds=(bf.GAUSS,), radii=(12,), orders=(24,), reps=2)
    assert len(entries) == 1 and 0 <= entries[0]["variant"] < bf.variant_count()
    tuning.save(entries, str(tmp_path / "t.json"))
    assert tuning.load(str(tmp_path / "t.json")) == 1
    img = image(60, 300, seed=21)
    out, q = bf.gpa_forward(torch.from_numpy(img).cuda(), bf.GAUSS, 30.0, 24, radius=12,
                            sigma_s=4.0, return_q=True)
    w = spatial(bf.GAUSS, 12, 4.0)
    ro, P, Q = oracle.gpa_alg2(img, w, 30.0, 24, return_parts=True)
    compare_forward(out.cpu().numpy(), q.cpu().numpy(), ro, scaled_q(img, Q, 30.0), w[12, 12],
                    "tuned", sigma_r=30.0, N=24, img=img, w=w)
    # the table's winner is the kernel the default call ran
    again = bf.gpa_forward(torch.from_numpy(img).cuda(), bf.GAUSS, 30.0, 24, radius=12,
                           sigma_s=4.0, variant=entries[0]["variant"])
    assert torch.equal(again, out)


@pytest.mark.gpu
@needs_gpu
def test_batch_autotuner_sets_entries_the_plan_follows(restored_table):
    """tuning.autotune_batch tunes the batch's buckets on its graph time; the
    plan built afterwards runs the table's variants, bitwise equal to the
    single-image calls with those variants."""
    from paper_1603_08109_gb300 import synth
    specs = synth.batch_specs(6, seed=31, max_hw=(200, 260))
    for sp in specs:
        sp["N"] = bf.order_from_delta(sp["kind"], sp["radius"], sp["sigma_s"], sp["sigma_r"], 1.0)
    imgs = [torch.from_numpy(image(sp["height"], sp["width"], seed=sp["seed"])).cuda()
            for sp in specs]
    outs = [torch.empty_like(x) for x in imgs]
    entries, before, after = tuning.autotune_batch(imgs, outs, specs, reps=2, coverage=1.0)
    assert entries and after <= before
    keys = {(e["kind"], e["radius_bucket"], e["order_bucket"]) for e in entries}
    assert keys == {(sp["kind"], bf.radius_bucket(sp["radius"]), bf.order_bucket(sp["N"]))
                    for sp in specs}
    for e in entries:
        assert bf.tuning_get(e["kind"], e["radius_bucket"], e["order_bucket"]) == e["variant"]
    plan = bf.BatchPlan(imgs, outs, specs)
    variants = plan.variants()
    plan.run()
    torch.cuda.synchronize()
    for x, o, sp, v in zip(imgs, outs, specs, variants):
        ref = bf.gpa_forward(x, sp["kind"], sp["sigma_r"], sp["N"], radius=sp["radius"],
                             sigma_s=sp["sigma_s"], variant=v)
        assert torch.equal(o, ref)
    plan.close()
