"""The allocation-free measurement entry point, through the C ABI.

micsa_measure_noalloc serves callers that must not allocate device memory
(their framework's allocator owns it all, or an allocation's implicit
synchronisation would stall a serving loop): they pass their own device arrays
and get the sums through a fixed scratch array inside the library. Here its
results are compared with micsa_measure on the same state, exactly (the sums
are integers), on two calls in a row -- the second after the state has moved
on, so a scratch array that kept the first call's sums would show.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

import paper_2506_16240_gb300 as micsa

pytestmark = pytest.mark.gpu


def _device_copies(torch, g):
    s, m, _ = g.get_state()
    J = g.get_couplings()
    dev = torch.device("cuda", torch.cuda.current_device())
    return (torch.from_numpy(s).to(dev), torch.from_numpy(m).to(dev), torch.from_numpy(J).to(dev))


@pytest.mark.parametrize("L,S,R", [(8, 1, 2), (16, 3, 4), (30, 2, 1)])
def test_noalloc_measure_matches_measure_twice(L, S, R):
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    stream = torch.cuda.Stream()
    with micsa.Micsa(L, S, R, 123 + L, stream=stream) as g:
        for call in range(2):
            g.run(np.linspace(2.5, 0.8, 37), 5)
            e_ref, a_ref, q_ref = g.measure()
            s_d, m_d, J_d = _device_copies(torch, g)
            torch.cuda.synchronize()
            e, a, q = micsa.measure_noalloc(s_d.data_ptr(), m_d.data_ptr(), J_d.data_ptr(), L, S, R,
                                            stream.cuda_stream)
            np.testing.assert_array_equal(e, e_ref, err_msg=f"energy, call {call}")
            np.testing.assert_array_equal(a, a_ref, err_msg=f"aux, call {call}")
            np.testing.assert_array_equal(q, q_ref, err_msg=f"overlap, call {call}")


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    # 32 replicas: 2*32 + 496 = 560 sums per sample; 15 samples need 8400 > 8192
    L, S, R = 2, 15, 32
    dev = torch.device("cuda", torch.cuda.current_device())
    s = torch.ones((S, R, L ** 3), dtype=torch.int8, device=dev)
    J = torch.ones((S, L ** 3, 3), dtype=torch.int8, device=dev)
    with pytest.raises(micsa.MicsaError) as err:
        micsa.measure_noalloc(s.data_ptr(), None, J.data_ptr(), L, S, R)
    assert err.value.code == micsa.MICSA_E_TOO_LARGE
    # 14 samples fit (7840 sums): all-up spins on all-ferro bonds give H = -3N
    e, a, q = micsa.measure_noalloc(s.data_ptr(), None, J.data_ptr(), L, 14, R)
    assert (e == -3 * L ** 3).all() and (a == 0).all() and (q == L ** 3).all()
