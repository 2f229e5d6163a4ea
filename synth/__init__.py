"""Seeded synthetic input generators (no transform arithmetic lives here)."""
from .inputs import *  # noqa: F401,F403
