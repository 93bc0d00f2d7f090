"""The allocation-free measurement entry point, through the C ABI.

micsa_measure_noalloc serves callers that must not allocate device memory
(their framework's allocator owns it all, or an allocation's implicit
synchronisation would stall a serving loop): they pass their own device arrays
and get the sums through a fixed scratch array inside the library. Its results
are compared exactly (the sums are integers) with micsa_measure and with the
CPU oracle on the same state, on two calls in a row -- the second after the
state has moved on, so a scratch array that kept the first call's sums would
show. Odd L, which micsa_create rejects but this entry point accepts, is checked
against the oracle on states written from the host.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

import oracle
import paper_2506_16240_gb300 as micsa

pytestmark = pytest.mark.gpu

O = oracle.Oracle()


def _oracle_sums(L, S, R, J, s, m):
    st = {"L": L, "S": S, "R": R, "J": np.ascontiguousarray(J, np.int8),
          "s": np.ascontiguousarray(s, np.int8), "m": np.ascontiguousarray(m, np.uint8)}
    return O.measure(st)


@pytest.mark.parametrize("L,S,R", [(8, 1, 2), (16, 3, 4), (30, 2, 1)])
def test_noalloc_measure_matches_measure_and_oracle_twice(L, S, R):
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    stream = torch.cuda.Stream()
    dev = torch.device("cuda", torch.cuda.current_device())
    with micsa.Micsa(L, S, R, 123 + L, stream=stream) as g:
        J = g.get_couplings()
        J_d = torch.from_numpy(J).to(dev)
        for call in range(2):
            g.run(np.linspace(2.5, 0.8, 37), 5)
            e_ref, a_ref, q_ref = g.measure()
            s, m, _ = g.get_state()
            s_d, m_d = torch.from_numpy(s).to(dev), torch.from_numpy(m).to(dev)
            torch.cuda.synchronize()
            e, a, q = micsa.measure_noalloc(s_d.data_ptr(), m_d.data_ptr(), J_d.data_ptr(), L, S, R,
                                            stream.cuda_stream)
            np.testing.assert_array_equal(e, e_ref, err_msg=f"energy, call {call}")
            np.testing.assert_array_equal(a, a_ref, err_msg=f"aux, call {call}")
            np.testing.assert_array_equal(q, q_ref, err_msg=f"overlap, call {call}")
            e_o, a_o, q_o = _oracle_sums(L, S, R, J.reshape(S, -1, 3), s, m)
            np.testing.assert_array_equal(e, e_o, err_msg=f"energy vs oracle, call {call}")
            np.testing.assert_array_equal(a, a_o, err_msg=f"aux vs oracle, call {call}")
            np.testing.assert_array_equal(q, q_o, err_msg=f"overlap vs oracle, call {call}")


@pytest.mark.parametrize("L,S,R", [(3, 2, 3), (5, 1, 2), (7, 3, 1)])
def test_noalloc_odd_lattices_match_oracle(L, S, R):
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    dev = torch.device("cuda", torch.cuda.current_device())
    rng = np.random.default_rng(1000 + L)
    N = L ** 3
    for call in range(2):
        J = np.where(rng.random((S, N, 3)) < 0.5, 1, -1).astype(np.int8)
        s = np.where(rng.random((S, R, N)) < 0.5, 1, -1).astype(np.int8)
        m = rng.integers(0, 4, (S, R, N)).astype(np.uint8)
        s_d, m_d, J_d = (torch.from_numpy(v).to(dev) for v in (s, m, J))
        torch.cuda.synchronize()
        e, a, q = micsa.measure_noalloc(s_d.data_ptr(), m_d.data_ptr(), J_d.data_ptr(), L, S, R)
        e_o, a_o, q_o = _oracle_sums(L, S, R, J, s, m)
        np.testing.assert_array_equal(e, e_o, err_msg=f"energy, call {call}")
        np.testing.assert_array_equal(a, a_o, err_msg=f"aux, call {call}")
        np.testing.assert_array_equal(q, q_o, err_msg=f"overlap, call {call}")


def test_noalloc_rejects_sizes_beyond_its_limits():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    # 32 replicas: 2*32 + 496 = 560 sums per sample; 15 samples need 8400 > 8192
    L, S, R = 2, 15, 32
    dev = torch.device("cuda", torch.cuda.current_device())
    s = torch.ones((S, R + 1, L ** 3), dtype=torch.int8, device=dev)
    J = torch.ones((S, L ** 3, 3), dtype=torch.int8, device=dev)
    with pytest.raises(micsa.MicsaError) as err:
        micsa.measure_noalloc(s.data_ptr(), None, J.data_ptr(), L, S, R)
    assert err.value.code == micsa.MICSA_E_TOO_LARGE
    # more than 32 replicas is outside the stated limits
    with pytest.raises(micsa.MicsaError) as err:
        micsa.measure_noalloc(s.data_ptr(), None, J.data_ptr(), L, 1, R + 1)
    assert err.value.code == micsa.MICSA_E_INVALID_ARG
    # 14 samples fit (7840 sums): all-up spins on all-ferro bonds give H = -3N
    s = torch.ones((14, R, L ** 3), dtype=torch.int8, device=dev)
    e, a, q = micsa.measure_noalloc(s.data_ptr(), None, J.data_ptr(), L, 14, R)
    assert (e == -3 * L ** 3).all() and (a == 0).all() and (q == L ** 3).all()
