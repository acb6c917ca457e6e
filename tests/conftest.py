"""Test configuration: the `gpu` marker and the import path.

Tests marked `gpu` need a CUDA device and the compiled engine library; every
other test runs on the CPU only.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled engine")
