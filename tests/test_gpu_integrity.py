"""Integrity of checkpoint images on restore (a corrupted or truncated image
must be reported, never replayed): the image manifest equals the oracle's
digests of the image's buffers, a restore verified against it gives the
oracle's result when the image is intact, and reports PHOS_ECORRUPT with
the lowest damaged buffer when a byte of the pinned image was changed on the
host; a truncated image is refused.  Every round mode."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import core  # noqa: E402
from oracle import protocols as P  # noqa: E402
from paper_2405_12079_b300 import phos, runner, workloads as wl  # noqa: E402


def a256(x):
    return (int(x) + 255) // 256 * 256


def world(seed):
    cfg = wl.training(scale=0.002, seed=seed, n_kernels=60)
    lay = cfg["layout"]
    rng = np.random.default_rng(seed)
    mem0 = np.zeros(lay.arena_bytes, np.uint8)
    wl.fill_random(rng, mem0)
    arena = torch.from_numpy(mem0.copy()).cuda()
    va0 = arena.data_ptr()
    ks = wl.make_training_kernels(rng, lay, va0, 60, cfg["n_rec"], 0.0)
    dp = runner.DeviceProcess(lay, arena, seed, ks)
    proc = P.Process(va0, lay.off, lay.size, mem0.copy(), seed)
    return lay, arena, ks, dp, proc


def manifest(dp, img):
    d = torch.zeros(8 * dp.layout.n, dtype=torch.uint8, device="cuda")
    phos.image_manifest(dp.table, img.data_ptr(), img.numel(), d.data_ptr(), dp.stream())
    torch.cuda.synchronize()
    return d


@pytest.mark.parametrize("rounds", ["sync", "nosync", "concurrent", "deferred"])
def test_verified_restore(rounds):
    lay, arena, ks, dp, proc = world(wl.SEED0 + 31)
    image = P.stw_checkpoint(proc)
    img = torch.from_numpy(image.copy()).pin_memory()
    d_man = manifest(dp, img)
    exp_dig = [core.digest(image[int(o):int(o) + int(sz)]) for o, sz in zip(dp.img_off, lay.size)]
    assert d_man.cpu().numpy().view(np.uint64).tolist() == exp_dig
    quota, chunk = a256(dp.image_bytes / 80), 64 * 1024

    # intact image: verified restore == the oracle's restore + replay
    arena.fill_(0xA5)
    cur = P.Process(dp.va0, lay.off, lay.size, np.full(lay.arena_bytes, 0xA5, np.uint8), proc.seed)
    exp = P.concurrent_restore(cur, image, ks, chunk, quota,
                               copier_stream=rounds in ("concurrent", "deferred"))
    got = dp.run_restore(img, quota, chunk, rounds=rounds, d_manifest=d_man)
    torch.cuda.synchronize()
    assert got["stats"]["corrupt_buf"] == -1 and got["stats"]["misspec_round"] == -1
    assert len(exp.ondemand) > 0
    assert np.array_equal(arena.cpu().numpy(), cur.mem)

    # two bytes of the pinned image changed on the host: buffers 137 and 600
    bad = (137, 600)
    for b in bad:
        img[int(dp.img_off[b]) + int(lay.size[b]) // 2] ^= 0x5A
    arena.fill_(0xA5)
    r = phos.Restore(dp.table, img.data_ptr(), img.numel(), chunk, 4, None, dp.stream(),
                     runner.DeviceProcess._flags(rounds), d_man.data_ptr())
    # the first call that synchronises after a damaged buffer landed
    # reports it (in lockstep rounds an after_kernel, else finish)
    with pytest.raises(phos.PhosError) as e:
        for k, pk in enumerate(dp.kernels):
            if r.advance(quota):
                break
            r.before_kernel(pk.speculate(dp.table, dp.perm))
            dp.run_kernel(k)
            r.after_kernel(pk.d_trace.data_ptr(), pk.n_rec)
        r.finish()
    assert e.value.code == phos.PHOS_ECORRUPT
    assert r.stats()["corrupt_buf"] in bad
    r.close()
    torch.cuda.synchronize()


def test_truncated_image_is_refused():
    lay, arena, ks, dp, proc = world(wl.SEED0 + 32)
    img = torch.from_numpy(P.stw_checkpoint(proc)).pin_memory()
    d_man = manifest(dp, img)
    short = dp.image_bytes - 256
    with pytest.raises(phos.PhosError) as e:
        phos.Restore(dp.table, img.data_ptr(), short, 64 * 1024, 4, None, dp.stream(), 0,
                     d_man.data_ptr())
    assert e.value.code == phos.PHOS_ECORRUPT
    with pytest.raises(phos.PhosError) as e:
        phos.image_manifest(dp.table, img.data_ptr(), short, d_man.data_ptr(), dp.stream())
    assert e.value.code == phos.PHOS_ECORRUPT
    # without a manifest a short image stays an argument error
    with pytest.raises(phos.PhosError) as e:
        phos.Restore(dp.table, img.data_ptr(), short, 64 * 1024, 4, None, dp.stream())
    assert e.value.code == phos.PHOS_EINVAL
