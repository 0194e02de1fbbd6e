import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def vocab_words():
    import synth
    return synth.make_vocab()


@pytest.fixture(scope="session")
def vocab_index(vocab_words):
    from oracle.tokenizer import build_vocab_index
    return build_vocab_index(vocab_words)


@pytest.fixture(scope="session")
def c1_records(vocab_words):
    import synth
    return synth.make_records(synth.C1.records, vocab_words)
