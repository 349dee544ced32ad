"""Device-allocation failures, injected on the host (tg_inject_alloc_failures):
every allocating call returns TG_ENOMEM at whichever of its allocations
fails, frees what it had allocated (the device's free memory is the same
before and after), and the library works normally once injection is off.
No GPU fault is involved: the injected failure never reaches the allocator."""
import pytest
import torch

pytestmark = pytest.mark.gpu

TG_ENOMEM = 2


def free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def fails_cleanly(tg, call, max_allocs=16):
    """Fails each allocation of `call` in turn; returns how many allocations the call makes."""
    before = free_bytes()
    for k in range(max_allocs):
        tg.tg_inject_alloc_failures(k, 1)
        try:
            obj = call()
        except tg.TGError as e:
            assert e.status == TG_ENOMEM, e
            assert "injected" in str(e)
            tg.tg_inject_alloc_failures(0, 0)
            assert free_bytes() == before, f"allocation {k} failed and left device memory behind"
            continue
        tg.tg_inject_alloc_failures(0, 0)
        del obj
        torch.cuda.synchronize()
        return k
    raise AssertionError("the call kept allocating")


def test_create_and_batch_fail_cleanly(tg):
    # load every kernel these calls launch first (module loading takes device memory once)
    warm = [tg.tg_create(3, 64, 2, 1, "f32"), tg.tg_create(3, 64, 2, 1, "bf16"), tg.tg_batch_create(3, 64, 1 << 16)]
    del warm
    try:
        assert fails_cleanly(tg, lambda: tg.tg_create(3, 64, 2, 1, "f32")) == 1        # master
        assert fails_cleanly(tg, lambda: tg.tg_create(3, 64, 2, 1, "bf16")) == 2       # master, stored copy
        assert fails_cleanly(tg, lambda: tg.tg_batch_create(3, 64, 1 << 16)) >= 6
    finally:
        tg.tg_inject_alloc_failures(0, 0)


def test_adam_state_and_query_binning_fail_cleanly(tg):
    P = torch.rand((1 << 20, 3), device="cuda")
    out = torch.empty((1 << 20, 1), device="cuda")
    warm = tg.tg_create(3, 64, 2, 1, "f32", seed=1, init_std=0.1)
    grad = torch.zeros(warm.n_coefs, device="cuda")
    tg.tg_adam_step(warm, grad, lr=1e-3, step=1)
    tg.tg_query(warm, P, out=out)
    del warm
    g = tg.tg_create(3, 64, 2, 1, "f32", seed=1, init_std=0.1)
    try:
        assert fails_cleanly(tg, lambda: tg.tg_adam_step(g, grad, lr=1e-3, step=1)) == 2     # m, v
        # a large 3-D tg_query bins into a grid-owned batch created on first use
        assert fails_cleanly(tg, lambda: tg.tg_query(g, P, out=out)) >= 6
    finally:
        tg.tg_inject_alloc_failures(0, 0)
    ref = tg.tg_query(g, P[:1000])          # the point-parallel path agrees with the binned one afterwards
    torch.testing.assert_close(out[:1000], ref, rtol=1e-5, atol=1e-6)
    assert tg.tg_grid_timeouts(g) == 0
