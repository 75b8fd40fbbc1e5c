"""Input generators: the valence transition matrix keeps exactly the functions of shells whose
largest primitive exponent is within the cut (no GPU)."""
import numpy as np

from paper_2512_18010_b300 import workloads as W


def test_valence_transitions_zero_exactly_the_core_functions():
    job = W.config3(3000)
    mol = job.mol
    Tv = W.valence_transitions(mol, job.T, 50.0)
    keep, off = [], 0
    for sh in range(mol.n_shells):
        npr = int(mol.shell_nprim[sh])
        keep += [float(np.max(mol.exponents[off:off + npr])) <= 50.0] * W.NFN[int(mol.shell_l[sh])]
        off += npr
    keep = np.array(keep)
    assert 0 < (~keep).sum() < keep.size                     # some core functions, most kept
    assert np.all(Tv[:, ~keep, :] == 0) and np.all(Tv[:, :, ~keep] == 0)
    kk = np.ix_(np.arange(job.n_states), keep, keep)
    assert np.array_equal(Tv[kk], job.T[kk])
    assert np.array_equal(W.valence_transitions(mol, job.T, 1e9), job.T)
