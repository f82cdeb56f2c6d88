"""B300-native per-invocation scheduling step of Llama (arXiv 2102.01887).

The package is imported lazily: ``workloads`` (seeded synthetic inputs) needs
only numpy, while ``llama`` loads the CUDA shared library on first use and
raises if it is missing.
"""
