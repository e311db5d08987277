"""bin_rays_static: the binning entry point for callers that cannot allocate
device memory (a host whose device memory all belongs to its own fixed pool,
or one with no device allocator to give bin_rays a workspace from).  It must
give exactly what bin_rays gives, call after call, although every call reuses
the same static device scratch and finds the previous call's data in it.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest

from paper_2405_06997_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2405_06997_gb300 import wfpg as W  # noqa: E402

KEYS = ("bin_of_ray", "ray_order", "bin_offset", "origin_ray", "n_bins")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def same(a, b):
    nb = int(a["n_bins"].item())
    assert nb == int(b["n_bins"].item())
    for k in ("bin_of_ray", "ray_order"):
        assert torch.equal(a[k], b[k]), k
    assert torch.equal(a["bin_offset"][: nb + 1], b["bin_offset"][: nb + 1])
    assert torch.equal(a["origin_ray"][:nb], b["origin_ray"][:nb])


def test_static_scratch_matches_workspace_version_twice():
    w = inputs.tiny_box(4, n_rays=5003)
    svo = W.svo_from_scene(w.scene, w.depth)
    pos, nrm = dev(w.ray_pos), dev(w.ray_nrm)
    # call 1: Partition-S
    a = W.bin_rays_static(svo, pos, l_min=2, c_ray=64, seed=3, frame=1)
    b = W.bin_rays(svo, pos, l_min=2, c_ray=64, seed=3, frame=1)
    torch.cuda.synchronize()
    same(a, b)
    # call 2: run mode on other rays, over the scratch call 1 left behind
    w2 = inputs.tiny_box(8, n_rays=7001)
    sizes = dev(inputs.zipf_bin_sizes(7001, 97, 1.2, 5).view(np.int32))
    pos2, nrm2 = dev(w2.ray_pos), dev(w2.ray_nrm)
    a = W.bin_rays_static(svo, pos2, nrm2, mode=W.BIN_RUNS, sizes=sizes, seed=2, frame=4)
    b = W.bin_rays(svo, pos2, nrm2, mode=W.BIN_RUNS, sizes=sizes, seed=2, frame=4)
    torch.cuda.synchronize()
    same(a, b)
    # call 3: Partition-S again, now after a run-mode call
    a = W.bin_rays_static(svo, pos, l_min=3, c_ray=16, seed=9, frame=2)
    b = W.bin_rays(svo, pos, l_min=3, c_ray=16, seed=9, frame=2)
    torch.cuda.synchronize()
    same(a, b)
    assert svo.status() == 0


def test_static_scratch_calls_allocate_nothing():
    """With its outputs allocated up front and one warm-up call made (the
    library's kernels loaded), further calls leave the device's free memory
    and torch's allocated bytes unchanged."""
    w = inputs.tiny_box(6, n_rays=6007)
    svo = W.svo_from_scene(w.scene, w.depth)
    pos = dev(w.ray_pos)
    n = pos.shape[0]
    bin_cap = max(1, min(n, svo.n_nodes))
    out = dict(bin_of_ray=torch.empty(n, dtype=torch.int32, device="cuda"),
               ray_order=torch.empty(n, dtype=torch.int32, device="cuda"),
               bin_offset=torch.empty(bin_cap + 1, dtype=torch.int32, device="cuda"),
               origin_ray=torch.empty(bin_cap, dtype=torch.int32, device="cuda"),
               n_bins=torch.zeros(1, dtype=torch.int32, device="cuda"))
    W.bin_rays_static(svo, pos, l_min=2, c_ray=32, seed=1, frame=0, bin_cap=bin_cap, out=out)
    torch.cuda.synchronize()
    free0, torch0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for k in range(3):
        W.bin_rays_static(svo, pos, l_min=2, c_ray=32, seed=1, frame=k + 1, bin_cap=bin_cap, out=out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == torch0
    assert svo.status() == 0


def test_static_scratch_rejects_calls_that_do_not_fit():
    w = inputs.tiny_box(4, n_rays=10)
    svo = W.svo_from_scene(w.scene, w.depth)
    n = 3_000_000   # RUNS mode needs ~12.3 B per ray: more than the 32 MiB scratch
    pos = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    sizes = torch.tensor([n], dtype=torch.int32, device="cuda")
    with pytest.raises(W.WfpgError) as e:
        W.bin_rays_static(svo, pos, pos, mode=W.BIN_RUNS, sizes=sizes)
    assert e.value.code == -5
    assert "static scratch" in str(e.value)
