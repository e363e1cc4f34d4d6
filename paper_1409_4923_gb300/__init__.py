"""GB300 (sm_103a) engine for Monte Carlo integration of Brownian-motor Langevin
equations with the jump-adapted simplified weak-order-2.0 predictor-corrector
scheme (Spiechowicz, Kostur & Machura, arXiv:1409.4923).

Importing the package loads nothing; `engine.lib()` loads libsde.so on first
use and raises if it is missing (there is no CPU fallback).
"""
__all__ = ["engine", "workloads"]
