"""Out-of-bounds writes, checked without compute-sanitizer: every device buffer of a context comes
through the allocator hook with 4 KiB guard zones of a known byte pattern on both sides; after a
run that crosses checkpoints and uses probes, the stream function, moments and population
exchange, every guard must be intact.  Odd sizes put wall columns, padding and ragged row groups
at every position a launch shape can see."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2211_05009_gb300 import binding as B  # noqa: E402
from paper_2211_05009_gb300.cavity import Cavity  # noqa: E402

GUARD = 4096
PATTERN = 0xA5


class GuardedAllocator:
    def __init__(self):
        self.live, self.bad = {}, []
        self.alloc_fn = B.ALLOC_FN(self._alloc)
        self.release_fn = B.RELEASE_FN(self._release)

    def _alloc(self, nbytes, user):
        body = (int(nbytes) + 255) // 256 * 256
        buf = torch.full((GUARD + body + GUARD,), PATTERN, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        p = buf.data_ptr() + GUARD
        self.live[p] = (buf, body)
        return p

    def check(self, p):
        buf, body = self.live[p]
        torch.cuda.synchronize()
        head, tail = buf[:GUARD], buf[GUARD + body:]
        if not (bool((head == PATTERN).all()) and bool((tail == PATTERN).all())):
            self.bad.append((p, body))

    def _release(self, ptr, user):
        if ptr in self.live:
            self.check(ptr)
            del self.live[ptr]


@pytest.mark.parametrize("nx,ny,dtype", [(5, 3, "f64"), (33, 9, "f32s"), (7, 130, "f32"), (37, 7, "f16s"),
                                         (129, 41, "bf16s"), (66, 9, "f64"), (131, 13, "q16s")])
def test_no_write_outside_any_buffer(nx, ny, dtype):
    ga = GuardedAllocator()
    B.lbm_set_allocator(ga.alloc_fn, ga.release_fn)
    try:
        with Cavity(nx, ny, Re=2.0 * nx, U=0.1, dtype=dtype) as cav:  # tau = 0.65 at every size
            assert ga.live, "the context allocates through the hook"
            q, series = cav.probe(0.5, 0.3, every=3, cap=40)
            cav.step(37)
            cav.step(213)  # crosses checkpoints 100 and 200 (graph replays and single steps)
            cav.residual()
            cav.stream_function(psi=True)
            rho, ux, uy = cav.moments()
            cav.set_moments(rho, ux, uy, neq=True)
            f = cav.populations()
            cav.set_populations(f)
            cav.step(120)
            cav.residual()
            for p in list(ga.live):
                ga.check(p)
    finally:
        B.lbm_set_allocator(None, None)
    assert not ga.live, "every buffer is released"
    assert not ga.bad, f"guard bytes changed next to {len(ga.bad)} buffer(s)"
    assert np.isfinite(series.cpu().numpy()).all()


def test_guard_check_detects_a_changed_byte():
    """The detector itself: a byte changed in a tail guard (written by torch, inside the guarded
    buffer) is reported; untouched buffers are not."""
    ga = GuardedAllocator()
    p1 = ga._alloc(1000, None)
    p2 = ga._alloc(3000, None)
    buf, body = ga.live[p1]
    buf[GUARD + body + 17] = 0
    ga._release(p1, None)
    ga._release(p2, None)
    assert ga.bad == [(p1, body)]
