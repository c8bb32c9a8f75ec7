"""Comparison arms that are neither the product nor the oracle (plain form)."""
